// Many queries against many resident tables of uneven sizes and widths in one
// persistent launch (the batched form of Sec. 3.2.1 extended across tables),
// and CUDA-graph capture of that launch.
//
// The planner groups each table's queries by eights and cuts the table into
// row ranges of 2^r rows, one work item per (range, group).  With an explicit
// item_log2 every table gets the same rows per item where it can (2^item_log2,
// clipped to the table), so items cost about the same and the kernel's item
// counter balances the rest; with item_log2 = 0 each table's r comes from the
// fused planner's cost model for its own queries (few queries: larger items).
// Items of one table range are adjacent, so the items in flight at any moment
// share table rows through L2.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

struct pir_multi_plan {
    int device = -1;
    uint32_t batch = 0;
    uint32_t item_log2 = 0;
    bool vec = true;
    std::vector<uint64_t> key_off, out_off;
    uint64_t key_total = 0, out_total = 0, nitems = 0;
    pir::MultiTable* d_tables = nullptr;
    pir::MultiItem* d_items = nullptr;
    uint64_t* d_key_off = nullptr;
    uint64_t* d_out_off = nullptr;
    uint64_t* d_counter = nullptr;
    uint8_t* d_stage_keys = nullptr;  // host-buffer entry point staging, allocated on first use
    uint32_t* d_stage_out = nullptr;
};

struct pir_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace pir {
namespace {

void free_plan(pir_multi_plan* p) {
    if (!p) return;
    cudaFree(p->d_tables);
    cudaFree(p->d_items);
    cudaFree(p->d_key_off);
    cudaFree(p->d_out_off);
    cudaFree(p->d_counter);
    cudaFree(p->d_stage_keys);
    cudaFree(p->d_stage_out);
    delete p;
}

template <typename T>
int upload(T** dst, const std::vector<T>& src) {
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return cuda_fail((int)e, "multi plan alloc");
    if (!src.empty()) {
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail((int)e, "multi plan upload");
    }
    return PIR_OK;
}

}  // namespace

int describe_tables(const pir_table* tables, size_t ntables, uint32_t item_log2, MultiLayout& lay) {
    const int G = multi_group();
    const int rmax = multi_max_range_log2();
    lay.auto_range = item_log2 == 0;
    if (item_log2 == 0) item_log2 = (uint32_t)rmax;
    if ((int)item_log2 > rmax) return PIR_ERR_UNSUPPORTED;
    lay.tables.assign(ntables, MultiTable{});
    lay.vec = true;
    for (size_t t = 0; t < ntables; ++t) {
        const pir_table& tb = tables[t];
        if (!tb.data || tb.rows < 1 || tb.width < 1 || tb.stride < tb.width ||
            (reinterpret_cast<uintptr_t>(tb.data) & 3u) != 0)
            return PIR_ERR_ARG;
        if ((uint64_t)G * tb.width > 4096u) return PIR_ERR_UNSUPPORTED;
        const uint32_t n = pir_domain_bits(tb.rows);
        if (n == 0) return PIR_ERR_DOMAIN;
        lay.vec = lay.vec && (reinterpret_cast<uintptr_t>(tb.data) & 15u) == 0 && tb.stride % 4 == 0 &&
                  tb.width % 4 == 0;
        MultiTable& m = lay.tables[t];
        m.data = tb.data;
        m.rows = tb.rows;
        m.stride = tb.stride;
        m.width = tb.width;
        m.n = n;
        m.key_bytes = (uint32_t)key_bytes(n);
        m.range_log2 = std::min<uint32_t>(n, item_log2);
    }
    // the kernel's consumers cover a row in W / VEC column chunks; with 32-bit
    // loads (some table not 16-byte aligned) that caps the width lower
    const uint32_t vec = lay.vec ? 4u : 1u;
    for (const MultiTable& m : lay.tables)
        if (m.width / vec > kFusedConsumerThreads) return PIR_ERR_UNSUPPORTED;
    return PIR_OK;
}

int plan_items(const uint32_t* table_of_key, size_t batch, MultiLayout& lay) {
    const int G = multi_group();
    const size_t ntables = lay.tables.size();
    lay.key_off.resize(batch);
    lay.out_off.resize(batch);
    lay.key_total = lay.out_total = 0;
    lay.items.clear();
    std::vector<std::vector<uint32_t>> per_table(ntables);
    for (size_t q = 0; q < batch; ++q) {
        const uint32_t t = table_of_key[q];
        if (t >= ntables) return PIR_ERR_ARG;
        lay.key_off[q] = lay.key_total;
        lay.out_off[q] = lay.out_total;
        lay.key_total += lay.tables[t].key_bytes;
        lay.out_total += lay.tables[t].width;
        per_table[t].push_back((uint32_t)q);
    }
    for (size_t t = 0; t < ntables; ++t) {
        const auto& qs = per_table[t];
        if (qs.empty()) continue;
        if (lay.auto_range) {
            // the table's largest slot count bounds its rows per item (a subtree is at
            // most kMaxDfsDepth levels deep); the cost model picks within that bound
            uint32_t gmax = 1;
            while (gmax < (uint32_t)G && gmax < qs.size()) gmax <<= 1;
            lay.tables[t].range_log2 = (uint32_t)plan_range_log2(
                lay.tables[t].rows, lay.tables[t].n, gmax, (uint32_t)((qs.size() + G - 1) / G));
        }
        const uint64_t ranges = ((lay.tables[t].rows - 1) >> lay.tables[t].range_log2) + 1;
        for (uint64_t rg = 0; rg < ranges; ++rg) {
            // groups of G queries; a last, smaller group gets the smallest power of two
            // of slots that holds it, so its item spreads over all of the CTA's producers
            for (size_t first = 0; first < qs.size(); first += (size_t)G) {
                const size_t left = std::min<size_t>((size_t)G, qs.size() - first);
                uint32_t g = 1;
                while (g < left) g <<= 1;
                MultiItem it{};
                it.table = (uint32_t)t;
                it.group = g;
                it.range = rg;
                for (int s = 0; s < 8; ++s) it.q[s] = ((uint32_t)s < g && (size_t)s < left) ? qs[first + s] : kNoQuery;
                lay.items.push_back(it);
            }
        }
    }
    return PIR_OK;
}

}  // namespace pir

extern "C" {

int pir_multi_plan_inspect(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                           uint32_t item_log2, pir_work_item* items, size_t capacity, uint64_t* nitems) {
    using namespace pir;
    if (!tables || ntables == 0 || ntables > 0xffffffffu || !table_of_key || batch == 0 || batch > 0xfffffffeu ||
        !nitems)
        return PIR_ERR_ARG;
    MultiLayout lay;
    int rc = describe_tables(tables, ntables, item_log2, lay);
    if (rc == PIR_OK) rc = plan_items(table_of_key, batch, lay);
    if (rc != PIR_OK) return rc;
    *nitems = lay.items.size();
    if (items) {
        for (size_t i = 0; i < lay.items.size() && i < capacity; ++i) {
            const MultiItem& m = lay.items[i];
            pir_work_item& w = items[i];
            w.table = m.table;
            w.group = m.group;
            w.range_log2 = lay.tables[m.table].range_log2;
            w.pad = 0;
            w.range = m.range;
            for (int q = 0; q < 8; ++q) w.query[q] = m.q[q];
        }
    }
    return PIR_OK;
}

int pir_multi_plan_create(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                          uint32_t item_log2, pir_multi_plan** out_plan) {
    using namespace pir;
    if (!tables || ntables == 0 || ntables > 0xffffffffu || !table_of_key || batch == 0 || batch > 0xfffffffeu ||
        !out_plan)
        return PIR_ERR_ARG;
    *out_plan = nullptr;
    MultiLayout lay;
    int rc = describe_tables(tables, ntables, item_log2, lay);
    if (rc == PIR_OK) rc = plan_items(table_of_key, batch, lay);
    if (rc != PIR_OK) return rc;
    pir_multi_plan* plan = new (std::nothrow) pir_multi_plan();
    if (!plan) return PIR_ERR_NOMEM;
    plan->batch = (uint32_t)batch;
    plan->item_log2 = item_log2;
    plan->vec = lay.vec;
    cudaGetDevice(&plan->device);
    plan->key_off = std::move(lay.key_off);
    plan->out_off = std::move(lay.out_off);
    plan->key_total = lay.key_total;
    plan->out_total = lay.out_total;
    plan->nitems = lay.items.size();
    rc = upload(&plan->d_tables, lay.tables);
    if (rc == PIR_OK) rc = upload(&plan->d_items, lay.items);
    if (rc == PIR_OK) rc = upload(&plan->d_key_off, plan->key_off);
    if (rc == PIR_OK) rc = upload(&plan->d_out_off, plan->out_off);
    if (rc == PIR_OK) {
        cudaError_t e = cudaMalloc((void**)&plan->d_counter, sizeof(uint64_t));
        if (e != cudaSuccess) rc = cuda_fail((int)e, "multi plan counter");
    }
    if (rc != PIR_OK) {
        free_plan(plan);
        return rc;
    }
    *out_plan = plan;
    return PIR_OK;
}

void pir_multi_plan_destroy(pir_multi_plan* plan) { pir::free_plan(plan); }

int pir_multi_plan_layout(const pir_multi_plan* plan, uint64_t* key_offsets, uint64_t* out_offsets,
                          uint64_t* key_bytes_total, uint64_t* out_words_total, uint64_t* items) {
    if (!plan) return PIR_ERR_ARG;
    if (key_offsets) std::memcpy(key_offsets, plan->key_off.data(), plan->batch * sizeof(uint64_t));
    if (out_offsets) std::memcpy(out_offsets, plan->out_off.data(), plan->batch * sizeof(uint64_t));
    if (key_bytes_total) *key_bytes_total = plan->key_total;
    if (out_words_total) *out_words_total = plan->out_total;
    if (items) *items = plan->nitems;
    return PIR_OK;
}

int pir_server_eval_multi(const pir_multi_plan* plan, const uint8_t* dkeys, uint32_t* dout, uint32_t* dstatus,
                          void* stream) {
    using namespace pir;
    if (!plan || !dkeys || !dout || (reinterpret_cast<uintptr_t>(dkeys) & 15u) != 0) return PIR_ERR_ARG;
    NvtxRange range("pir_server_eval_multi");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(dout, 0, plan->out_total * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->d_counter, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail((int)e, "multi memset");
    MultiParams mp{};
    mp.tables = plan->d_tables;
    mp.items = plan->d_items;
    mp.nitems = plan->nitems;
    mp.key_off = plan->d_key_off;
    mp.out_off = plan->d_out_off;
    mp.keys = dkeys;
    mp.out = dout;
    mp.status = dstatus;
    mp.counter = plan->d_counter;
    return launch_multi(mp, plan->vec, stream);
}

int pir_server_eval_multi_host(pir_multi_plan* plan, const uint8_t* keys, uint32_t* out, void* stream) {
    using namespace pir;
    if (!plan || !keys || !out) return PIR_ERR_ARG;
    NvtxRange range("pir_server_eval_multi_host");
    if (!plan->d_stage_keys) {
        cudaError_t e = cudaMalloc((void**)&plan->d_stage_keys, std::max<uint64_t>(16, plan->key_total));
        if (e == cudaSuccess)
            e = cudaMalloc((void**)&plan->d_stage_out, std::max<uint64_t>(1, plan->out_total) * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail((int)e, "multi staging alloc");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(plan->d_stage_keys, keys, plan->key_total, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail((int)e, "multi copy keys");
    int rc = pir_server_eval_multi(plan, plan->d_stage_keys, plan->d_stage_out, nullptr, stream);
    if (rc != PIR_OK) return rc;
    e = cudaMemcpyAsync(out, plan->d_stage_out, plan->out_total * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "multi copy shares");
}

int pir_multi_graph_create(const pir_multi_plan* plan, const uint8_t* dkeys, uint32_t* dout, uint32_t* dstatus,
                           pir_graph** out_graph) {
    using namespace pir;
    if (!plan || !out_graph) return PIR_ERR_ARG;
    *out_graph = nullptr;
    pir_graph* g = new (std::nothrow) pir_graph();
    if (!g) return PIR_ERR_NOMEM;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail((int)e, "graph stream");
    }
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? PIR_OK : cuda_fail((int)e, "begin capture");
    if (rc == PIR_OK) {
        rc = pir_server_eval_multi(plan, dkeys, dout, dstatus, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
        if (rc == PIR_OK && e2 != cudaSuccess) rc = cuda_fail((int)e2, "end capture");
    }
    if (rc == PIR_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail((int)e, "graph instantiate");
    }
    cudaStreamDestroy(s);
    if (rc != PIR_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc;
    }
    *out_graph = g;
    return PIR_OK;
}

int pir_graph_launch(pir_graph* g, void* stream) {
    if (!g || !g->exec) return PIR_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PIR_OK : pir::cuda_fail((int)e, "graph launch");
}

void pir_graph_destroy(pir_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int pir_multi_autotune(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                       const uint8_t* dkeys, uint32_t* dout, void* stream, uint32_t* best_item_log2,
                       float* best_ms) {
    using namespace pir;
    if (!best_item_log2) return PIR_ERR_ARG;
    NvtxRange range("pir_multi_autotune");
    const int rmax = multi_max_range_log2();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 0.f;
    uint32_t best_r = 0;
    int rc = PIR_OK;
    for (int r = rmax; r >= rmax - 4 && r >= 8; --r) {
        pir_multi_plan* plan = nullptr;
        rc = pir_multi_plan_create(tables, ntables, table_of_key, batch, (uint32_t)r, &plan);
        if (rc != PIR_OK) break;
        rc = pir_server_eval_multi(plan, dkeys, dout, nullptr, stream);  // warm-up
        float ms = 0.f;
        if (rc == PIR_OK) {
            cudaEventRecord(a, s);
            for (int i = 0; i < 3 && rc == PIR_OK; ++i) rc = pir_server_eval_multi(plan, dkeys, dout, nullptr, stream);
            cudaEventRecord(b, s);
            cudaError_t e = cudaEventSynchronize(b);
            if (e != cudaSuccess && rc == PIR_OK) rc = cuda_fail((int)e, "autotune sync");
            cudaEventElapsedTime(&ms, a, b);
        }
        pir_multi_plan_destroy(plan);
        if (rc != PIR_OK) break;
        if (best_r == 0 || ms < best) {
            best = ms;
            best_r = (uint32_t)r;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != PIR_OK) return rc;
    *best_item_log2 = best_r;
    if (best_ms) *best_ms = best / 3.f;
    return PIR_OK;
}

}  // extern "C"
