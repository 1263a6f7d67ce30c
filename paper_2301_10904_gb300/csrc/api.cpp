// C-ABI server entry points: argument checks, buffer staging, dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"

namespace pir {

static thread_local char g_cuda_msg[256] = "no CUDA error";

int cuda_fail(int code, const char* what) {
    std::snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s (%d)", what, cudaGetErrorString((cudaError_t)code), code);
    return code == (int)cudaErrorMemoryAllocation ? PIR_ERR_NOMEM : PIR_ERR_CUDA;
}

#define CUDA_TRY(call, what)                                \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail((int)e_, what); \
    } while (0)

static bool table_ok(const pir_table* t) {
    return t && t->data && t->rows >= 1 && t->width >= 1 && t->stride >= t->width &&
           (reinterpret_cast<uintptr_t>(t->data) & 3u) == 0;
}

static bool vec_ok(const pir_table* t) {
    return (reinterpret_cast<uintptr_t>(t->data) & 15u) == 0 && t->stride % 4 == 0 && t->width % 4 == 0;
}

static bool is_device_pointer(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // unregistered host memory on older runtimes
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- staging memory for the host-buffer entry points ---------------------
// Stream-ordered allocations from a pool the library owns (one per device).
// The pool keeps up to kStagingKeepBytes of freed blocks mapped across stream
// synchronisations; the device's default pool would hand them back to the
// driver at every synchronisation and map them again on the next call.
constexpr uint64_t kStagingKeepBytes = 256ull << 20;
constexpr int kMaxDevices = 64;

int staging_pool(cudaMemPool_t* pool) {
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "get device");
    if (dev < 0 || dev >= kMaxDevices) return PIR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        CUDA_TRY(cudaMemPoolCreate(&p, &props), "create staging pool");
        uint64_t keep = kStagingKeepBytes;
        cudaError_t e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return cuda_fail((int)e, "staging pool threshold");
        }
        pools[dev] = p;
    }
    *pool = pools[dev];
    return PIR_OK;
}

// ---- autotuned launch shapes --------------------------------------------
// Keyed by (device, rows, width, batch rounded up to a power of two, whether
// 128-bit loads apply); filled by pir_autotune, read by every evaluation.
struct ShapeKey {
    int device;
    uint64_t rows;
    uint32_t width;
    uint32_t batch_bucket;
    bool vec;
    bool operator<(const ShapeKey& o) const {
        if (device != o.device) return device < o.device;
        if (rows != o.rows) return rows < o.rows;
        if (width != o.width) return width < o.width;
        if (batch_bucket != o.batch_bucket) return batch_bucket < o.batch_bucket;
        return vec < o.vec;
    }
};
static std::mutex g_tuned_mu;
static std::map<ShapeKey, pir_plan> g_tuned;

static ShapeKey shape_key(uint64_t rows, uint32_t width, size_t batch, bool vec) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t bucket = 1;
    while (bucket < batch && bucket < (1u << 30)) bucket <<= 1;
    return ShapeKey{dev, rows, width, bucket, vec};
}

static bool tuned_plan(uint64_t rows, uint32_t width, size_t batch, bool vec, pir_plan* out) {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    auto it = g_tuned.find(shape_key(rows, width, batch, vec));
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
}

// Runs the fused evaluation of rows [row_lo, row_lo + shard->rows) of a
// 2^n-leaf domain for device keys into a zeroed device output.
// One or two queries against a table whose rows are wide for the batch (at
// least kTwoPassRowWords words per query) and of at least kTwoPassMinBytes:
// expanding the share vectors into scratch (the level-by-level strategy, Sec.
// 3.2.2) and streaming the table once through the scan engine beats the fused
// kernel.  There each table row read serves one or two queries, and the fused
// consumers' loads queue behind the producers' table lookups in the SM's
// shared-memory pipe, so too few rows are in flight.  GB300, one query: 2^20 x
// 64 words 0.107 vs 0.130 ms, 2^22 x 64 0.366 vs 0.441, 2^24 x 64 1.33 vs 1.57,
// 2^19 x 128 0.086 vs 0.102; two queries, 2^20 x 128 0.200 vs 0.227.  With
// narrower rows the fused kernel wins: one query on 2^24 x 32 0.966 vs 1.028
// ms, 2^22 x 32 0.279 vs 0.292; two on 2^20 x 64 0.151 vs 0.159.  The scratch
// (rows x 4 bytes per query) comes from the staging pool.
constexpr uint64_t kTwoPassMinBytes = 128ull << 20;
constexpr uint32_t kTwoPassRowWords = 64;
static bool two_pass_preferred(uint64_t rows, uint32_t width, size_t batch) {
    return batch <= 2 && width >= kTwoPassRowWords * batch && rows * (uint64_t)width * 4u >= kTwoPassMinBytes;
}

static int eval_two_pass(const pir_table* t, uint32_t n, const uint8_t* dkeys, size_t batch, uint32_t* dout,
                         uint32_t* dstatus, void* stream) {
    NvtxRange range("pir: expand + scan");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t ld = (t->rows + 3) & ~3ull;
    cudaMemPool_t pool = nullptr;
    int rc = staging_pool(&pool);
    if (rc != PIR_OK) return rc;
    pir_plan plan{};
    rc = plan_fused(t->rows, 0, n, 1, (uint32_t)batch, false, &plan);
    if (rc != PIR_OK) return rc;
    uint32_t* S = nullptr;
    CUDA_TRY(cudaMallocFromPoolAsync((void**)&S, ld * batch * sizeof(uint32_t), pool, s), "alloc share vectors");
    EvalRequest req{};
    req.row_lo = 0;
    req.row_hi = t->rows;
    req.width = 1;
    req.stride = 1;
    req.n = n;
    req.dkeys = dkeys;
    req.batch = (uint32_t)batch;
    req.dstatus = dstatus;
    rc = launch_materialise(req, plan, S, ld, stream);
    if (rc == PIR_OK) {
        cudaError_t e = cudaMemsetAsync(dout, 0, batch * t->width * sizeof(uint32_t), s);
        rc = e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "memset shares");
    }
    if (rc == PIR_OK) rc = launch_scan(S, ld, (uint32_t)batch, t->data, t->stride, t->width, t->rows, dout, stream);
    cudaFreeAsync(S, s);
    return rc;
}

// The strategy and launch shape an evaluation of rows [row_lo, row_lo +
// shard->rows) of a 2^n-leaf domain runs: an explicit plan (checked), else the
// autotuned one for the shape, else the heuristic (expand + scan for one or two
// queries on wide rows, the fused kernel otherwise).  No device work.
static int resolve_plan(const pir_table* shard, uint64_t row_lo, uint32_t n, size_t batch, const pir_plan* plan_in,
                        pir_plan* out) {
    if (!table_ok(shard) || batch == 0 || batch > 0xffffffffu) return PIR_ERR_ARG;
    if (n == 0 || n > PIR_MAX_DOMAIN_BITS) return PIR_ERR_DOMAIN;
    if (row_lo + shard->rows > (1ull << n)) return PIR_ERR_DOMAIN;
    const bool v = vec_ok(shard);
    // the scan engine's layout (its scratch is 16-byte aligned with ld % 4 == 0)
    const bool two_ok = row_lo == 0 && v && shard->stride <= 1024;
    pir_plan plan{};
    if (plan_in) {
        plan = *plan_in;
        int rc = PIR_ERR_ARG;
        if (plan.strategy == PIR_STRATEGY_EXPAND_SCAN)
            rc = two_ok ? PIR_OK : PIR_ERR_UNSUPPORTED;
        else if (plan.strategy == PIR_STRATEGY_FUSED)
            rc = plan_check(plan, n, shard->width, v);
        else if (plan.strategy == PIR_STRATEGY_FUSED_STAGED)
            rc = plan_check_staged(plan, n, shard->width, shard->stride, v);
        if (rc != PIR_OK) return rc;
        *out = plan;
        return PIR_OK;
    }
    if (row_lo == 0 && tuned_plan(shard->rows, shard->width, batch, v, &plan)) {
        if (plan.strategy == PIR_STRATEGY_EXPAND_SCAN && two_ok) {
            *out = plan;
            return PIR_OK;
        }
        // tuned per power-of-two batch bucket: cut the last round for this batch
        plan.tail_log2 = plan_tail_log2(0, shard->rows, n, plan.group, (uint32_t)batch, plan.range_log2);
        if ((plan.strategy == PIR_STRATEGY_FUSED && plan_check(plan, n, shard->width, v) == PIR_OK) ||
            (plan.strategy == PIR_STRATEGY_FUSED_STAGED &&
             plan_check_staged(plan, n, shard->width, shard->stride, v) == PIR_OK)) {
            *out = plan;
            return PIR_OK;
        }
    }
    const int rc = plan_fused(shard->rows, row_lo, n, shard->width, (uint32_t)batch, v, &plan);
    if (rc != PIR_OK) return rc;
    if (two_ok && two_pass_preferred(shard->rows, shard->width, batch)) plan.strategy = PIR_STRATEGY_EXPAND_SCAN;
    *out = plan;
    return PIR_OK;
}

// Whether a strategy's kernels have bounded waits (mbarrier pipelines) that
// can give up and record PIR_FAULT_WAIT_TIMEOUT in the device fault word.
static bool strategy_waits(uint32_t strategy) {
    return strategy == PIR_STRATEGY_EXPAND_SCAN || strategy == PIR_STRATEGY_FUSED_STAGED;
}

// Runs a resolved plan for device keys into the device output (overwritten;
// `zeroed`: the caller knows it already holds zeros).
static int run_plan(const pir_table* shard, uint64_t row_lo, uint32_t n, const uint8_t* dkeys, size_t batch,
                    uint32_t* dout, uint32_t* dstatus, const pir_plan& plan, void* stream, bool zeroed = false) {
    if (plan.strategy == PIR_STRATEGY_EXPAND_SCAN) return eval_two_pass(shard, n, dkeys, batch, dout, dstatus, stream);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!zeroed) CUDA_TRY(cudaMemsetAsync(dout, 0, batch * shard->width * sizeof(uint32_t), s), "memset shares");
    EvalRequest req{};
    req.table = shard->data;
    req.row_lo = row_lo;
    req.row_hi = row_lo + shard->rows;
    req.width = shard->width;
    req.stride = shard->stride;
    req.n = n;
    req.dkeys = dkeys;
    req.batch = (uint32_t)batch;
    req.dout = dout;
    req.dstatus = dstatus;
    NvtxRange range("pir: fused launch");
    return launch_fused(req, plan, stream);
}

static int eval_device(const pir_table* shard, uint64_t row_lo, uint32_t n, const uint8_t* dkeys, size_t batch,
                       uint32_t* dout, uint32_t* dstatus, const pir_plan* plan_in, void* stream) {
    if (!table_ok(shard) || !dkeys || !dout || batch == 0 || batch > 0xffffffffu) return PIR_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(dkeys) & 15u) != 0) return PIR_ERR_ARG;
    pir_plan plan{};
    const int rc = resolve_plan(shard, row_lo, n, batch, plan_in, &plan);
    if (rc != PIR_OK) return rc;
    return run_plan(shard, row_lo, n, dkeys, batch, dout, dstatus, plan, stream);
}

// Staging of the synchronous host-buffer path, per host thread and device,
// for small calls (a lone query: the latency-bound case).  The keys and a
// zeroed share area are laid out in mapped pinned host memory as they will
// lie on the device and reach it in one copy; the call (that copy, the
// kernels, the copy of the shares back to mapped pinned memory) runs as a
// CUDA graph, built on the first call of its shape and kept, so that the GPU
// runs the steps back to back instead of waiting for each host API call.
// Both copies are small kernels reading and writing the host side directly,
// not copy-engine transfers, whose start-up dominated at these sizes.  A
// call returns only after its shares are on the host, so the buffers are
// idle when the next call of the thread starts.  Kept until the thread exits.
constexpr size_t kStageKeyBytes = 32u << 10, kStageShareBytes = 32u << 10;
constexpr size_t kStageBytes = kStageKeyBytes + 256 + kStageShareBytes;
constexpr size_t kStageGraphs = 8;  // graphs kept per thread and device (least recently used goes)

struct StageShape {  // what a staged call's graph depends on
    const uint32_t* table;
    uint64_t rows, stride, batch;
    uint32_t width, n;
    pir_plan plan;
    bool snap;
    bool operator==(const StageShape& o) const {
        return table == o.table && rows == o.rows && stride == o.stride && batch == o.batch && width == o.width &&
               n == o.n && snap == o.snap && plan.group == o.plan.group && plan.range_log2 == o.plan.range_log2 &&
               plan.vec == o.plan.vec && plan.ctas == o.plan.ctas && plan.strategy == o.plan.strategy &&
               plan.tail_log2 == o.plan.tail_log2;
    }
};

struct HostStage {
    uint8_t* dev = nullptr;   // device: keys, then the share area at a 256-byte boundary
    uint8_t* hin = nullptr;   // mapped pinned host: the same layout, copied to `dev` in one piece
    uint8_t* hout = nullptr;  // mapped pinned host: the shares copied back
    uint32_t *hin_dev = nullptr, *hout_dev = nullptr;  // their device addresses
    cudaStream_t capture = nullptr;
    cudaEvent_t done = nullptr;
    struct Graph {
        StageShape shape;
        cudaGraphExec_t exec;  // nullptr: this shape could not be captured (the pool path runs it)
        uint64_t used;
    };
    std::vector<Graph> graphs;
    uint64_t tick = 0;
    ~HostStage() {
        for (Graph& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (done) cudaEventDestroy(done);
        if (capture) cudaStreamDestroy(capture);
        if (hout) cudaFreeHost(hout);
        if (hin) cudaFreeHost(hin);
        if (dev) cudaFree(dev);
    }
    static size_t share_offset(size_t key_bytes) { return (key_bytes + 255) & ~size_t(255); }
};
static HostStage* host_stage() {
    thread_local HostStage stages[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    HostStage& st = stages[dev];
    if (!st.dev) {
        if (cudaMalloc((void**)&st.dev, kStageBytes) != cudaSuccess ||
            cudaHostAlloc((void**)&st.hin, kStageBytes, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void**)&st.hout, kStageShareBytes, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&st.hin_dev, st.hin, 0) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&st.hout_dev, st.hout, 0) != cudaSuccess ||
            cudaStreamCreateWithFlags(&st.capture, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (st.done) cudaEventDestroy(st.done);
            if (st.capture) cudaStreamDestroy(st.capture);
            if (st.hin) cudaFreeHost(st.hin);
            if (st.hout) cudaFreeHost(st.hout);
            if (st.dev) cudaFree(st.dev);
            st.done = nullptr;
            st.capture = nullptr;
            st.hin = st.hout = nullptr;
            st.hin_dev = st.hout_dev = nullptr;
            st.dev = nullptr;
            return nullptr;  // the caller takes the pool path
        }
    }
    return &st;
}

// The graph of a staged call of shape `sh` (keys of `kb` bytes each, shares of
// `out_bytes`), built on first use: the one copy of keys and zeroed shares to
// the device, the fault-word snapshots around the kernels when `snap` is
// given, the kernels, the shares' copy back.  nullptr when the shape could
// not be captured (the caller then takes the pool path; the answer is kept).
static cudaGraphExec_t stage_graph(HostStage& st, const StageShape& sh, const pir_table* t, size_t kb,
                                   size_t out_bytes, uint32_t* snap, uint32_t* fault_word) {
    for (HostStage::Graph& g : st.graphs)
        if (g.shape == sh) {
            g.used = ++st.tick;
            return g.exec;
        }
    const size_t ks = HostStage::share_offset(sh.batch * kb);
    uint32_t* dout = reinterpret_cast<uint32_t*>(st.dev + ks);
    cudaStream_t c = st.capture;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(c, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        bool ok = launch_words_copy(st.hin_dev, reinterpret_cast<uint32_t*>(st.dev), (ks + out_bytes) / 4, c) == PIR_OK;
        if (ok && snap)
            ok = cudaMemcpyAsync(&snap[0], fault_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, c) == cudaSuccess;
        if (ok) ok = run_plan(t, 0, sh.n, st.dev, sh.batch, dout, nullptr, sh.plan, c, /*zeroed=*/true) == PIR_OK;
        if (ok && snap)
            ok = cudaMemcpyAsync(&snap[1], fault_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, c) == cudaSuccess;
        if (ok) ok = launch_words_copy(dout, st.hout_dev, out_bytes / 4, c) == PIR_OK;
        const bool ended = cudaStreamEndCapture(c, &graph) == cudaSuccess;
        if (ok && ended && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a capture that failed leaves its error here, not for the caller's next call
    if (st.graphs.size() >= kStageGraphs) {
        auto lru = std::min_element(st.graphs.begin(), st.graphs.end(),
                                    [](const HostStage::Graph& a, const HostStage::Graph& b) { return a.used < b.used; });
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        st.graphs.erase(lru);
    }
    st.graphs.push_back({sh, exec, ++st.tick});
    return exec;
}

// Two words of pinned host memory per host thread, for stream-ordered
// snapshots of the device fault word (allocated on first use).
static uint32_t* fault_snapshots() {
    thread_local uint32_t* words = nullptr;
    if (!words && cudaHostAlloc((void**)&words, 2 * sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        words = nullptr;
    }
    return words;
}

}  // namespace pir

extern "C" {

const char* pir_error_string(int code) {
    switch (code) {
        case PIR_OK: return "ok";
        case PIR_ERR_ARG: return "invalid argument";
        case PIR_ERR_DOMAIN: return "key domain does not match the table";
        case PIR_ERR_KEY: return "malformed key";
        case PIR_ERR_NOMEM: return "out of memory";
        case PIR_ERR_CUDA: return "CUDA error";
        case PIR_ERR_TIMEOUT: return "timed out";
        case PIR_ERR_BUSY: return "busy";
        case PIR_ERR_UNSUPPORTED: return "unsupported shape";
        case PIR_ERR_CANCELLED: return "cancelled";
        default: return "unknown error";
    }
}

const char* pir_last_cuda_error(void) { return pir::g_cuda_msg; }

// The untuned choice of pir_server_eval_device for an aligned table of this shape on a device with `sms` SMs.
static int heuristic_plan(uint64_t rows, uint32_t width, size_t batch, int sms, pir_plan* plan) {
    if (!plan || rows < 1 || width == 0 || batch == 0 || batch > 0xffffffffu || sms < 1) return PIR_ERR_ARG;
    const uint32_t n = pir_domain_bits(rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const int rc = pir::plan_fused_sms(rows, 0, n, width, (uint32_t)batch, width % 4 == 0, sms, plan);
    if (rc == PIR_OK && width % 4 == 0 && width <= 1024 && pir::two_pass_preferred(rows, width, batch))
        plan->strategy = PIR_STRATEGY_EXPAND_SCAN;
    return rc;
}

int pir_plan_for(uint64_t rows, uint32_t width, size_t batch, pir_plan* plan) {
    if (!plan || rows < 1 || width == 0 || batch == 0 || batch > 0xffffffffu) return PIR_ERR_ARG;
    if (pir_domain_bits(rows) == 0) return PIR_ERR_DOMAIN;
    if (pir::tuned_plan(rows, width, batch, width % 4 == 0, plan)) return PIR_OK;
    return heuristic_plan(rows, width, batch, std::max(1, pir::device_sm_count()), plan);
}

int pir_plan_inspect(uint64_t rows, uint32_t width, size_t batch, uint32_t sms, pir_plan* plan) {
    if (sms == 0 || sms > 65536) return PIR_ERR_ARG;
    return heuristic_plan(rows, width, batch, (int)sms, plan);
}

int pir_plan_pin(const pir_table* t, size_t batch, const pir_plan* plan) {
    using namespace pir;
    if (!table_ok(t) || batch == 0 || batch > 0xffffffffu) return PIR_ERR_ARG;
    const uint32_t n = pir_domain_bits(t->rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const bool v = vec_ok(t);
    const ShapeKey key = shape_key(t->rows, t->width, batch, v);
    if (!plan) {
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        g_tuned.erase(key);
        return PIR_OK;
    }
    // the checks of an explicit plan (pir_server_eval_device_plan)
    pir_plan checked{};
    const int rc = resolve_plan(t, 0, n, batch, plan, &checked);
    if (rc != PIR_OK) return rc;
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_tuned[key] = checked;
    return PIR_OK;
}

int pir_autotune(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout, void* stream,
                 pir_plan* best_plan, float* best_ms) {
    using namespace pir;
    if (!table_ok(t) || !dkeys || !dout || batch == 0 || batch > 0xffffffffu || !best_plan) return PIR_ERR_ARG;
    NvtxRange range("pir_autotune");
    const uint32_t n = pir_domain_bits(t->rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const bool v = vec_ok(t);
    pir_plan base{};
    int rc = plan_fused(t->rows, 0, n, t->width, (uint32_t)batch, v, &base);
    if (rc != PIR_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    pir_plan best = base;
    float best_t = -1.f;
    for (uint32_t g = 8; g >= 1; g >>= 1) {
        if (g > batch || (uint64_t)g * t->width > 4096u) continue;
        for (int r = (int)n; r >= 1; --r) {
            pir_plan pl{g, (uint32_t)r, base.vec, 0};
            pl.tail_log2 = plan_tail_log2(0, t->rows, n, g, (uint32_t)batch, (uint32_t)r);
            if (plan_check(pl, n, t->width, v) != PIR_OK) continue;
            // keep shapes with at least one item per SM, or the whole table in one item
            const uint32_t nqg = (uint32_t)((batch + g - 1) / g);
            const uint64_t items = (((t->rows - 1) >> r) + 1) * nqg;
            if (items < (uint64_t)std::max(1, device_sm_count()) / 2 && r != (int)n && r > 8) continue;
            if (r + 6 < (int)base.range_log2) break;  // far below the heuristic: only more path walks
            // the fused kernel, and for small groups near the heuristic's rows per item
            // also its staged form (table rows through the shared-memory ring)
            for (uint32_t strat : {PIR_STRATEGY_FUSED, PIR_STRATEGY_FUSED_STAGED}) {
                pl.strategy = strat;
                if (strat == PIR_STRATEGY_FUSED_STAGED &&
                    (g > 4 || r + 1 < (int)base.range_log2 || r > (int)base.range_log2 ||
                     plan_check_staged(pl, n, t->width, t->stride, v) != PIR_OK))
                    continue;
                rc = eval_device(t, 0, n, dkeys, batch, dout, nullptr, &pl, stream);  // warm-up
                if (rc != PIR_OK) break;
                cudaEventRecord(a, s);
                for (int i = 0; i < 3 && rc == PIR_OK; ++i)
                    rc = eval_device(t, 0, n, dkeys, batch, dout, nullptr, &pl, stream);
                cudaEventRecord(b, s);
                cudaError_t e = cudaEventSynchronize(b);
                if (rc != PIR_OK) break;
                if (e != cudaSuccess) {
                    rc = cuda_fail((int)e, "autotune sync");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                ms /= 3.f;
                if (best_t < 0.f || ms < best_t) {
                    best_t = ms;
                    best = pl;
                }
            }
            if (rc != PIR_OK) break;
        }
        if (rc != PIR_OK) break;
        if (g == 1) break;
    }
    // the expand-and-scan strategy, where the scan engine takes this layout
    if (rc == PIR_OK && batch <= 8 && v && t->stride <= 1024) {
        rc = eval_two_pass(t, n, dkeys, batch, dout, nullptr, stream);  // warm-up
        if (rc == PIR_OK) {
            cudaEventRecord(a, s);
            for (int i = 0; i < 3 && rc == PIR_OK; ++i) rc = eval_two_pass(t, n, dkeys, batch, dout, nullptr, stream);
            cudaEventRecord(b, s);
            cudaError_t e = cudaEventSynchronize(b);
            if (rc == PIR_OK && e != cudaSuccess) rc = cuda_fail((int)e, "autotune sync");
            float ms = 0.f;
            if (rc == PIR_OK) cudaEventElapsedTime(&ms, a, b);
            ms /= 3.f;
            if (rc == PIR_OK && (best_t < 0.f || ms < best_t)) {
                best_t = ms;
                best = base;
                best.strategy = PIR_STRATEGY_EXPAND_SCAN;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != PIR_OK) return rc;
    const uint32_t nqg = (uint32_t)((batch + best.group - 1) / best.group);
    best.ctas = (uint32_t)std::min<uint64_t>((((t->rows - 1) >> best.range_log2) + 1) * nqg,
                                             (uint64_t)std::max(1, device_sm_count()));
    {
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        g_tuned[shape_key(t->rows, t->width, batch, v)] = best;
    }
    *best_plan = best;
    if (best_ms) *best_ms = best_t;
    return PIR_OK;
}

int pir_server_eval_device(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout, uint32_t* dstatus,
                           void* stream) {
    if (!t) return PIR_ERR_ARG;
    return pir::eval_device(t, 0, pir_domain_bits(t->rows), dkeys, batch, dout, dstatus, nullptr, stream);
}

int pir_server_eval_device_plan(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout,
                                uint32_t* dstatus, const pir_plan* plan, void* stream) {
    if (!t || !plan) return PIR_ERR_ARG;
    return pir::eval_device(t, 0, pir_domain_bits(t->rows), dkeys, batch, dout, dstatus, plan, stream);
}

int pir_server_eval_range(const pir_table* shard, uint64_t row_lo, uint64_t domain_rows, const uint8_t* dkeys,
                          size_t batch, uint32_t* dout, uint32_t* dstatus, void* stream) {
    if (!shard || domain_rows < 1 || row_lo + shard->rows > domain_rows) return PIR_ERR_ARG;
    return pir::eval_device(shard, row_lo, pir_domain_bits(domain_rows), dkeys, batch, dout, dstatus, nullptr, stream);
}

int pir_server_eval_pbr(const pir_table* t, uint64_t bin_rows, const uint8_t* dkeys, uint32_t* dout,
                        uint32_t* dstatus, void* stream) {
    using namespace pir;
    if (!table_ok(t) || !dkeys || !dout || bin_rows < 2) return PIR_ERR_ARG;
    NvtxRange range("pir_server_eval_pbr");
    if ((reinterpret_cast<uintptr_t>(dkeys) & 15u) != 0) return PIR_ERR_ARG;
    if (!vec_ok(t)) return PIR_ERR_UNSUPPORTED;
    const uint32_t n = pir_domain_bits(bin_rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const uint64_t nbins = (t->rows + bin_rows - 1) / bin_rows;
    if (nbins > 0xffffffffull) return PIR_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        // one launch: each CTA expands its bins' trees, then multiplies its own rows
        const int rc = launch_pbr_fused(t->data, t->rows, t->width, t->stride, bin_rows, n, dkeys, (uint32_t)nbins,
                                        dout, dstatus, stream);
        if (rc != PIR_ERR_UNSUPPORTED) return rc;
    }
    if (scan_bins_supported(t->data, t->stride, t->width, bin_rows)) {
        // two passes: every bin's share vector into scratch (one word per table row,
        // nbins x bin_rows words from the staging pool), then one streaming pass over
        // the table in which each chunk of rows multiplies its own bin's shares
        // (1.5-2x the fused bins kernel on GB300, whose product side cannot keep
        // enough loads in flight when no row is shared between queries)
        cudaMemPool_t pool = nullptr;
        int rc = staging_pool(&pool);
        if (rc != PIR_OK) return rc;
        pir_plan plan{};
        rc = plan_fused(bin_rows, 0, n, 1, (uint32_t)nbins, false, &plan);
        if (rc != PIR_OK) return rc;
        uint32_t* S = nullptr;
        CUDA_TRY(cudaMallocFromPoolAsync((void**)&S, nbins * bin_rows * sizeof(uint32_t), pool, s), "alloc bin shares");
        EvalRequest req{};
        req.row_lo = 0;
        req.row_hi = bin_rows;
        req.width = 1;
        req.stride = 1;
        req.n = n;
        req.dkeys = dkeys;
        req.batch = (uint32_t)nbins;
        req.dstatus = dstatus;
        rc = launch_materialise(req, plan, S, bin_rows, stream);
        if (rc == PIR_OK) {
            cudaError_t e = cudaMemsetAsync(dout, 0, nbins * t->width * sizeof(uint32_t), s);
            rc = e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "memset shares");
        }
        if (rc == PIR_OK) rc = launch_scan_bins(S, t->data, t->stride, t->width, t->rows, bin_rows, dout, stream);
        cudaFreeAsync(S, s);
        return rc;
    }
    pir_plan plan{};
    int rc = plan_bins(bin_rows, n, t->width, (uint32_t)nbins, &plan);
    if (rc != PIR_OK) return rc;
    CUDA_TRY(cudaMemsetAsync(dout, 0, nbins * t->width * sizeof(uint32_t), s), "memset shares");
    EvalRequest req{};
    req.table = t->data;
    req.row_lo = 0;
    req.row_hi = t->rows;
    req.width = t->width;
    req.stride = t->stride;
    req.n = n;
    req.dkeys = dkeys;
    req.batch = (uint32_t)nbins;
    req.dout = dout;
    req.dstatus = dstatus;
    return launch_bins(req, bin_rows, plan, stream);
}

int pir_expand_materialise(uint64_t rows, const uint8_t* dkeys, size_t batch, uint32_t* dshares, uint64_t ld,
                           uint32_t* dstatus, void* stream) {
    using namespace pir;
    if (!dkeys || !dshares || batch == 0 || batch > 0xffffffffu || rows < 1 || ld < rows) return PIR_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(dkeys) & 15u) != 0 || (reinterpret_cast<uintptr_t>(dshares) & 3u) != 0)
        return PIR_ERR_ARG;
    const uint32_t n = pir_domain_bits(rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    pir_plan plan{};
    int rc = plan_fused(rows, 0, n, 1, (uint32_t)batch, false, &plan);
    if (rc != PIR_OK) return rc;
    EvalRequest req{};
    req.row_lo = 0;
    req.row_hi = rows;
    req.width = 1;
    req.stride = 1;
    req.n = n;
    req.dkeys = dkeys;
    req.batch = (uint32_t)batch;
    req.dstatus = dstatus;
    return launch_materialise(req, plan, dshares, ld, stream);
}

int pir_staging_stats(uint64_t* reserved_bytes, uint64_t* used_bytes) {
    using namespace pir;
    if (!reserved_bytes || !used_bytes) return PIR_ERR_ARG;
    cudaMemPool_t pool = nullptr;
    const int rc = staging_pool(&pool);
    if (rc != PIR_OK) return rc;
    uint64_t reserved = 0, used = 0;
    CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved), "staging pool reserved");
    CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used), "staging pool used");
    *reserved_bytes = reserved;
    *used_bytes = used;
    return PIR_OK;
}

int pir_selftest_bounded_wait(uint32_t polls, void* stream) {
    if (polls == 0) return PIR_ERR_ARG;
    return pir::selftest_bounded_wait(polls, stream);
}

int pir_device_status(uint32_t* flags, int clear) {
    if (!flags) return PIR_ERR_ARG;
    return pir::device_faults(flags, clear != 0);
}

int pir_contract_u32(const uint32_t* dshares, uint64_t ld, size_t batch, const pir_table* t, uint32_t* dout,
                     int engine, void* stream) {
    using namespace pir;
    if (!table_ok(t) || !dshares || !dout || batch == 0 || batch > 0xffffffffu || ld < t->rows) return PIR_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(dout, 0, batch * t->width * sizeof(uint32_t), s), "memset shares");
    return launch_contract(dshares, ld, (uint32_t)batch, t->data, t->stride, t->width, t->rows, dout, engine, stream);
}

int pir_server_eval(const pir_table* t, const uint8_t* keys, size_t batch, uint32_t* out, void* stream) {
    using namespace pir;
    NvtxRange range("pir_server_eval");
    if (!table_ok(t) || !keys || !out || batch == 0) return PIR_ERR_ARG;
    const uint32_t n = pir_domain_bits(t->rows);
    if (n == 0) return PIR_ERR_DOMAIN;
    const size_t kb = key_bytes(n);
    for (size_t q = 0; q < batch; ++q) {
        uint32_t kn = 0, party = 0;
        const uint8_t* k = keys + q * kb;
        // the length is implied by the table's domain: check the header fields
        int rc = pir_key_check(k, key_bytes(k[5] <= PIR_MAX_DOMAIN_BITS ? k[5] : 0), &kn, &party);
        if (rc != PIR_OK) return PIR_ERR_KEY;
        if (kn != n) return PIR_ERR_DOMAIN;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool out_on_device = is_device_pointer(out);
    const size_t out_bytes = batch * (size_t)t->width * sizeof(uint32_t);
    pir_plan plan{};
    int rc = resolve_plan(t, 0, n, batch, nullptr, &plan);
    if (rc != PIR_OK) return rc;
    // a strategy whose kernels have bounded waits: snapshot the device fault
    // word before and after it (stream-ordered), so that a wait that gave up
    // during this call turns into PIR_ERR_TIMEOUT once the call synchronizes
    uint32_t* snap = !out_on_device && strategy_waits(plan.strategy) ? fault_snapshots() : nullptr;
    uint32_t* fault_word = snap ? device_fault_word() : nullptr;
    if (!fault_word) snap = nullptr;
    cudaError_t e = cudaSuccess;
    HostStage* st = !out_on_device && batch * kb <= kStageKeyBytes && out_bytes <= kStageShareBytes &&
                            plan.strategy != PIR_STRATEGY_EXPAND_SCAN
                        ? host_stage()
                        : nullptr;
    if (st) {
        // the staged graph: keys and zeroed shares in pinned memory, one launch, shares back
        const size_t key_total = batch * kb, ks = HostStage::share_offset(key_total);
        std::memcpy(st->hin, keys, key_total);
        std::memset(st->hin + key_total, 0, ks - key_total + out_bytes);
        StageShape sh{t->data, t->rows, t->stride, batch, t->width, n, plan, snap != nullptr};
        cudaGraphExec_t exec = stage_graph(*st, sh, t, kb, out_bytes, snap, fault_word);
        if (exec) {
            e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(st->done, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(st->done);
            if (e != cudaSuccess) {
                rc = cuda_fail((int)e, "staged call");
                cudaStreamSynchronize(s);
                return rc;
            }
            std::memcpy(out, st->hout, out_bytes);
            if (snap && (snap[1] & ~snap[0] & PIR_FAULT_WAIT_TIMEOUT)) return PIR_ERR_TIMEOUT;
            return PIR_OK;
        }
    }
    // stream-ordered staging from the pool
    uint8_t* dkeys = nullptr;
    uint32_t* dout = nullptr;
    cudaMemPool_t pool = nullptr;
    rc = staging_pool(&pool);
    if (rc != PIR_OK) return rc;
    CUDA_TRY(cudaMallocFromPoolAsync((void**)&dkeys, batch * kb, pool, s), "alloc keys");
    if (!out_on_device) {
        e = cudaMallocFromPoolAsync((void**)&dout, out_bytes, pool, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(dkeys, s);
            return cuda_fail((int)e, "alloc shares");
        }
    } else {
        dout = out;
    }
    e = cudaMemcpyAsync(dkeys, keys, batch * kb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail((int)e, "copy keys");
    if (rc == PIR_OK && fault_word) {
        e = cudaMemcpyAsync(&snap[0], fault_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail((int)e, "fault word snapshot");
    }
    if (rc == PIR_OK) rc = run_plan(t, 0, n, dkeys, batch, dout, nullptr, plan, stream);
    if (rc == PIR_OK && fault_word) {
        e = cudaMemcpyAsync(&snap[1], fault_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail((int)e, "fault word snapshot");
    }
    if (rc == PIR_OK && !out_on_device) {
        e = cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail((int)e, "copy shares");
    }
    if (!out_on_device) cudaFreeAsync(dout, s);
    cudaFreeAsync(dkeys, s);
    if (!out_on_device) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess && rc == PIR_OK) rc = cuda_fail((int)e, "synchronize");
    }
    if (rc == PIR_OK && fault_word && (snap[1] & ~snap[0] & PIR_FAULT_WAIT_TIMEOUT)) rc = PIR_ERR_TIMEOUT;
    return rc;
}

}  // extern "C"
