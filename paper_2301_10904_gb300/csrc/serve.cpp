// Serving loop: continuous cross-table batching of PIR queries on one GPU.
//
// Requests (a key for one registered table) are admitted into a fixed pool of
// request slots whose size follows from a device-memory budget; a full pool
// refuses new requests with PIR_ERR_BUSY.  A worker thread forms a batch from
// everything pending (up to max_batch queries, any mix of tables), packs the
// keys and the multi-table work list into one pinned block, and launches
// copy-in, the persistent multi-table kernel and copy-out on one of several
// streams.  While a batch runs, requests that arrive meanwhile form the next
// batch on another stream, so their work overlaps on the device.  Tables stay
// resident; every request's latency is stamped from its arrival to the moment
// its share is in the caller's buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

enum ReqState : int { kFree = 0, kPending = 1, kRunning = 2, kDone = 3 };

struct Request {
    uint32_t gen = 0;
    int state = kFree;
    uint32_t table = 0;
    uint32_t key_len = 0;
    uint8_t key[PIR_KEY_HEADER_BYTES + 64 * PIR_MAX_DOMAIN_BITS];
    uint32_t* out = nullptr;        // caller's host buffer (width words)
    int64_t* latency_out = nullptr;  // optional
    bool detached = false;           // released by the worker when done (no poll)
    int64_t t_arrival = 0, t_done = 0;
    int status = PIR_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint32_t> reqs;       // request indices, batch order
    std::vector<uint64_t> out_off;    // word offset of each request's share
    uint8_t* d_block = nullptr;       // tables | items | key offsets | share offsets | keys
    uint8_t* h_block = nullptr;       // pinned mirror
    size_t block_cap = 0;
    uint32_t* d_out = nullptr;
    uint32_t* h_out = nullptr;        // pinned
    size_t out_cap = 0;               // words
    std::vector<void*> retired_host;  // outgrown pinned buffers, freed with the server
    uint64_t* d_counter = nullptr;
    uint32_t* d_status = nullptr;
};

}  // namespace

struct pir_server {
    pir_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_idle;
    std::vector<pir_table> tables;
    std::vector<Request> reqs;
    std::vector<uint32_t> free_list;
    std::deque<uint32_t> pending;
    uint32_t running = 0;  // requests in launched batches
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    int worker_error = PIR_OK;
    pir_server_stats stats{};
};

namespace pir {

// The library's stream-ordered allocation pool for the current device (api.cpp).
int staging_pool(cudaMemPool_t* pool);

namespace {

// Device buffer of `bytes` (stream-ordered, from the library's pool) and its
// pinned mirror, replacing (d, h) only when both allocations succeed.  The old
// device buffer is freed in stream order; the old pinned one is kept until the
// server is destroyed (freeing pinned memory synchronises the whole device,
// which would stall the batch in flight on the other streams).
int realloc_pair(Slot& s, cudaMemPool_t pool, size_t bytes, void** d, void** h) {
    void* nd = nullptr;
    void* nh = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&nd, bytes, pool, s.stream);
    if (e == cudaSuccess) e = cudaMallocHost(&nh, bytes);
    if (e != cudaSuccess) {
        if (nd) cudaFreeAsync(nd, s.stream);
        return cuda_fail((int)e, "serve buffer alloc");
    }
    if (*d) cudaFreeAsync(*d, s.stream);
    if (*h) s.retired_host.push_back(*h);
    *d = nd;
    *h = nh;
    return PIR_OK;
}

// Makes slot s hold a batch of block_bytes and out_words; counts reallocations.
// Slots are sized for a full batch when the server starts, so this is rare.
int grow(Slot& s, size_t block_bytes, size_t out_words, uint32_t* grown) {
    *grown = 0;
    if (block_bytes <= s.block_cap && out_words <= s.out_cap) return PIR_OK;
    cudaMemPool_t pool = nullptr;
    int rc = staging_pool(&pool);
    if (rc != PIR_OK) return rc;
    if (block_bytes > s.block_cap) {
        const size_t cap = std::max(block_bytes, s.block_cap * 2);
        rc = realloc_pair(s, pool, cap, (void**)&s.d_block, (void**)&s.h_block);
        if (rc != PIR_OK) return rc;
        s.block_cap = cap;
        ++*grown;
    }
    if (out_words > s.out_cap) {
        const size_t cap = std::max(out_words, s.out_cap * 2);
        rc = realloc_pair(s, pool, cap * 4, (void**)&s.d_out, (void**)&s.h_out);
        if (rc != PIR_OK) return rc;
        s.out_cap = cap;
        ++*grown;
    }
    return PIR_OK;
}

// Worker side: finished batches hand their shares to the requests.
void retire(pir_server* srv, Slot& s) {
    NvtxRange range("serve: retire batch");
    const int64_t t = now_ns();
    std::lock_guard<std::mutex> lock(srv->mu);
    for (size_t i = 0; i < s.reqs.size(); ++i) {
        Request& r = srv->reqs[s.reqs[i]];
        const uint32_t w = srv->tables[r.table].width;
        std::memcpy(r.out, s.h_out + s.out_off[i], w * sizeof(uint32_t));
        r.t_done = t;
        if (r.latency_out) *r.latency_out = t - r.t_arrival;
        if (r.detached) {
            r.state = kFree;
            ++r.gen;
            srv->free_list.push_back(s.reqs[i]);
        } else {
            r.state = kDone;
        }
    }
    srv->running -= (uint32_t)s.reqs.size();
    srv->stats.completed += s.reqs.size();
    s.reqs.clear();
    s.busy = false;
    srv->cv_idle.notify_all();
}

// Worker side: a batch that could not run, or failed on the device, ends its
// requests with error `rc` (their callers see it from pir_poll / the replay).
void fail_batch(pir_server* srv, const std::vector<uint32_t>& batch, int rc) {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->worker_error = rc;
    for (uint32_t id : batch) {
        Request& r = srv->reqs[id];
        r.status = rc;
        r.t_done = now_ns();
        if (r.latency_out) *r.latency_out = -1;
        if (r.detached) {
            r.state = kFree;
            ++r.gen;
            srv->free_list.push_back(id);
        } else {
            r.state = kDone;
        }
    }
    srv->running -= (uint32_t)batch.size();
    srv->cv_idle.notify_all();
}

// Worker side: packs and launches one batch on slot s.
int launch_batch(pir_server* srv, Slot& s, const std::vector<uint32_t>& batch, const std::vector<pir_table>& tables,
                 MultiLayout& lay) {
    NvtxRange range("serve: plan, pack and launch batch");
    std::vector<uint32_t> table_of_key(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) table_of_key[i] = srv->reqs[batch[i]].table;
    int rc = describe_tables(tables.data(), tables.size(), srv->cfg.item_log2, lay);
    if (rc == PIR_OK) rc = plan_items(table_of_key.data(), batch.size(), lay);
    if (rc != PIR_OK) return rc;
    const size_t o_tab = 0;
    const size_t o_items = align16(o_tab + lay.tables.size() * sizeof(MultiTable));
    const size_t o_koff = align16(o_items + lay.items.size() * sizeof(MultiItem));
    const size_t o_ooff = align16(o_koff + batch.size() * sizeof(uint64_t));
    const size_t o_keys = align16(o_ooff + batch.size() * sizeof(uint64_t));
    const size_t total = align16(o_keys + lay.key_total);
    uint32_t grown = 0;
    rc = grow(s, total, lay.out_total, &grown);
    if (grown) {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stats.grows += grown;
    }
    if (rc != PIR_OK) return rc;
    std::memcpy(s.h_block + o_tab, lay.tables.data(), lay.tables.size() * sizeof(MultiTable));
    std::memcpy(s.h_block + o_items, lay.items.data(), lay.items.size() * sizeof(MultiItem));
    std::memcpy(s.h_block + o_koff, lay.key_off.data(), batch.size() * sizeof(uint64_t));
    std::memcpy(s.h_block + o_ooff, lay.out_off.data(), batch.size() * sizeof(uint64_t));
    for (size_t i = 0; i < batch.size(); ++i) {
        const Request& r = srv->reqs[batch[i]];
        std::memcpy(s.h_block + o_keys + lay.key_off[i], r.key, r.key_len);
    }
    s.out_off = lay.out_off;
    cudaError_t e = cudaMemcpyAsync(s.d_block, s.h_block, total, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_out, 0, lay.out_total * sizeof(uint32_t), s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_counter, 0, sizeof(uint64_t), s.stream);
    if (e != cudaSuccess) return cuda_fail((int)e, "serve copy-in");
    MultiParams mp{};
    mp.tables = reinterpret_cast<const MultiTable*>(s.d_block + o_tab);
    mp.items = reinterpret_cast<const MultiItem*>(s.d_block + o_items);
    mp.nitems = lay.items.size();
    mp.key_off = reinterpret_cast<const uint64_t*>(s.d_block + o_koff);
    mp.out_off = reinterpret_cast<const uint64_t*>(s.d_block + o_ooff);
    mp.keys = s.d_block + o_keys;
    mp.out = s.d_out;
    mp.status = s.d_status;
    mp.counter = s.d_counter;
    rc = launch_multi(mp, lay.vec, s.stream);
    if (rc != PIR_OK) return rc;
    e = cudaMemcpyAsync(s.h_out, s.d_out, lay.out_total * sizeof(uint32_t), cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    if (e != cudaSuccess) return cuda_fail((int)e, "serve copy-out");
    s.reqs = batch;
    s.busy = true;
    return PIR_OK;
}

void worker_main(pir_server* srv) {
    cudaSetDevice(srv->device);
    MultiLayout lay;
    std::vector<pir_table> tables;
    std::vector<uint32_t> batch;
    for (;;) {
        bool progressed = false;
        for (Slot& s : srv->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaSuccess) {
                retire(srv, s);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                // the batch failed on the device: its requests end with an error, not a hang
                fail_batch(srv, s.reqs, cuda_fail((int)q, "serve batch"));
                s.reqs.clear();
                s.busy = false;
                progressed = true;
            }
        }
        Slot* free_slot = nullptr;
        for (Slot& s : srv->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        batch.clear();
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            bool any_busy = false;
            for (Slot& s : srv->slots) any_busy = any_busy || s.busy;
            if (srv->stop && srv->pending.empty() && !any_busy) return;
            if (free_slot && !srv->pending.empty()) {
                while (!srv->pending.empty() && batch.size() < srv->cfg.max_batch) {
                    const uint32_t id = srv->pending.front();
                    srv->pending.pop_front();
                    srv->reqs[id].state = kRunning;
                    batch.push_back(id);
                }
                srv->running += (uint32_t)batch.size();
                tables = srv->tables;
            } else if (!progressed) {
                // nothing to retire or launch: wait for work, or poll running batches
                srv->cv_work.wait_for(lock, std::chrono::microseconds(any_busy ? 10 : 200));
                continue;
            }
        }
        if (!batch.empty()) {
            const int rc = launch_batch(srv, *free_slot, batch, tables, lay);
            if (rc != PIR_OK) {
                // the batch cannot run: fail its requests rather than hang their callers
                fail_batch(srv, batch, rc);
            } else {
                std::lock_guard<std::mutex> lock(srv->mu);
                srv->stats.batches += 1;
                srv->stats.batched_queries += batch.size();
            }
        }
    }
}

uint64_t make_ticket(uint32_t gen, uint32_t idx) { return ((uint64_t)gen << 32) | idx; }

int submit(pir_server* srv, uint32_t table_id, const uint8_t* key, uint32_t* out, int64_t t_arrival,
           int64_t* latency_out, bool detached, uint64_t* ticket) {
    if (!srv || !key || !out) return PIR_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) return PIR_ERR_ARG;
    if (table_id >= srv->tables.size()) return PIR_ERR_ARG;
    const uint32_t n = pir_domain_bits(srv->tables[table_id].rows);
    uint32_t kn = 0, party = 0;
    // the header's own n gives the key's length; a valid key of another domain is a domain error
    if (pir_key_check(key, key_bytes(key[5] <= PIR_MAX_DOMAIN_BITS ? key[5] : 0), &kn, &party) != PIR_OK)
        return PIR_ERR_KEY;
    if (kn != n) return PIR_ERR_DOMAIN;
    if (srv->free_list.empty()) {
        srv->stats.rejected += 1;
        return PIR_ERR_BUSY;
    }
    const uint32_t id = srv->free_list.back();
    srv->free_list.pop_back();
    Request& r = srv->reqs[id];
    r.state = kPending;
    r.table = table_id;
    r.key_len = (uint32_t)key_bytes(n);
    std::memcpy(r.key, key, r.key_len);
    r.out = out;
    r.latency_out = latency_out;
    r.detached = detached;
    r.t_arrival = t_arrival;
    r.t_done = 0;
    r.status = PIR_OK;
    srv->pending.push_back(id);
    srv->stats.submitted += 1;
    if (ticket) *ticket = make_ticket(r.gen, id);
    srv->cv_work.notify_one();
    return PIR_OK;
}

}  // namespace
}  // namespace pir

extern "C" {

int pir_server_create(const pir_server_config* cfg_in, pir_server** out) {
    using namespace pir;
    if (!out) return PIR_ERR_ARG;
    *out = nullptr;
    pir_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_batch == 0) cfg.max_batch = 2048;
    if (cfg.streams == 0) cfg.streams = 2;
    if (cfg.streams > 8) return PIR_ERR_ARG;
    if (cfg.device_memory_budget == 0) cfg.device_memory_budget = 256ull << 20;
    if (cfg.max_inflight == 0) {
        // per admitted query: its key (<= 2,592 B), a share of up to 512 words, and its share of work items
        const uint64_t per_query = 2592 + 2048 + 64 * sizeof(MultiItem);
        cfg.max_inflight = (uint32_t)std::min<uint64_t>(1u << 20, cfg.device_memory_budget / per_query);
    }
    if (cfg.max_inflight == 0) return PIR_ERR_NOMEM;
    pir_server* srv = new (std::nothrow) pir_server();
    if (!srv) return PIR_ERR_NOMEM;
    srv->cfg = cfg;
    cudaGetDevice(&srv->device);
    srv->reqs.resize(cfg.max_inflight);
    srv->free_list.reserve(cfg.max_inflight);
    for (uint32_t i = cfg.max_inflight; i-- > 0;) srv->free_list.push_back(i);
    srv->slots.resize(cfg.streams);
    int rc = PIR_OK;
    for (Slot& s : srv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_counter, sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_status, sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemset(s.d_status, 0, sizeof(uint32_t));
        if (e != cudaSuccess) {
            rc = cuda_fail((int)e, "serve slot");
            break;
        }
        // a full batch: up to 64 table descriptors; per query up to 256 work items
        // (the planner gives a lone query about one item per SM, 128 on 152 SMs;
        // queries of one table share items), a key of the widest domain and two
        // offsets; and 512 share words per query
        const size_t block = align16(64 * sizeof(MultiTable)) +
                             (size_t)cfg.max_batch * (256 * sizeof(MultiItem) + 2 * sizeof(uint64_t) + 2592);
        uint32_t grown = 0;
        rc = grow(s, block, (size_t)cfg.max_batch * 512, &grown);
        if (rc == PIR_OK) {
            const cudaError_t se = cudaStreamSynchronize(s.stream);
            if (se != cudaSuccess) rc = cuda_fail((int)se, "serve slot sync");
        }
        if (rc != PIR_OK) break;
    }
    if (rc != PIR_OK) {
        pir_server_destroy(srv);
        return rc;
    }
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return PIR_OK;
}

int pir_server_register_table(pir_server* srv, const pir_table* t, uint32_t* table_id) {
    using namespace pir;
    if (!srv || !t || !t->data || t->rows < 1 || t->width < 1 || t->width > 512 || t->stride < t->width || !table_id)
        return PIR_ERR_ARG;
    if (pir_domain_bits(t->rows) == 0) return PIR_ERR_DOMAIN;
    std::lock_guard<std::mutex> lock(srv->mu);
    *table_id = (uint32_t)srv->tables.size();
    srv->tables.push_back(*t);
    return PIR_OK;
}

int pir_submit(pir_server* srv, uint32_t table_id, const uint8_t* key, uint32_t* out, uint64_t* ticket) {
    return pir::submit(srv, table_id, key, out, now_ns(), nullptr, false, ticket);
}

int pir_poll(pir_server* srv, uint64_t ticket, int64_t* latency_ns) {
    if (!srv) return PIR_ERR_ARG;
    const uint32_t idx = (uint32_t)ticket, gen = (uint32_t)(ticket >> 32);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (idx >= srv->reqs.size()) return PIR_ERR_ARG;
    Request& r = srv->reqs[idx];
    if (r.gen != gen || r.state == kFree || r.detached) return PIR_ERR_ARG;
    if (r.state != kDone) return PIR_ERR_BUSY;
    if (latency_ns) *latency_ns = r.t_done - r.t_arrival;
    const int status = r.status;
    r.state = kFree;
    ++r.gen;
    srv->free_list.push_back(idx);
    return status;
}

int pir_cancel(pir_server* srv, uint64_t ticket) {
    if (!srv) return PIR_ERR_ARG;
    const uint32_t idx = (uint32_t)ticket, gen = (uint32_t)(ticket >> 32);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (idx >= srv->reqs.size()) return PIR_ERR_ARG;
    Request& r = srv->reqs[idx];
    if (r.gen != gen || r.state == kFree || r.detached) return PIR_ERR_ARG;
    if (r.state != kPending) return PIR_ERR_BUSY;  // already in a batch, or done
    auto it = std::find(srv->pending.begin(), srv->pending.end(), idx);
    if (it == srv->pending.end()) return PIR_ERR_BUSY;
    srv->pending.erase(it);
    r.state = kFree;
    r.status = PIR_ERR_CANCELLED;
    ++r.gen;
    srv->free_list.push_back(idx);
    srv->stats.cancelled += 1;
    srv->cv_idle.notify_all();
    return PIR_OK;
}

int pir_server_drain(pir_server* srv, uint32_t timeout_ms) {
    if (!srv) return PIR_ERR_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    const bool ok = srv->cv_idle.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                          [&] { return srv->pending.empty() && srv->running == 0; });
    if (!ok) return PIR_ERR_TIMEOUT;
    return srv->worker_error;
}

int pir_server_stats_get(pir_server* srv, pir_server_stats* st) {
    if (!srv || !st) return PIR_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    *st = srv->stats;
    st->max_inflight = srv->cfg.max_inflight;
    return PIR_OK;
}

int pir_server_replay(pir_server* srv, const double* arrival_s, const uint32_t* table_ids, const uint8_t* keys,
                      const uint64_t* key_offsets, size_t count, uint32_t* outs, const uint64_t* out_offsets,
                      int64_t* latency_ns, double* elapsed_s) {
    if (!srv || !arrival_s || !table_ids || !keys || !key_offsets || !outs || !out_offsets || !latency_ns)
        return PIR_ERR_ARG;
    const int64_t t0 = now_ns();
    for (size_t i = 0; i < count; ++i) {
        const int64_t due = t0 + (int64_t)(arrival_s[i] * 1e9);
        while (now_ns() < due) std::this_thread::yield();
        for (;;) {  // a full pool makes the client wait; its latency keeps counting from `due`
            const int rc = pir::submit(srv, table_ids[i], keys + key_offsets[i], outs + out_offsets[i], due,
                                       &latency_ns[i], true, nullptr);
            if (rc == PIR_OK) break;
            if (rc != PIR_ERR_BUSY) return rc;
            std::this_thread::sleep_for(std::chrono::microseconds(5));
        }
    }
    const int rc = pir_server_drain(srv, 600000);
    if (elapsed_s) *elapsed_s = (double)(now_ns() - t0) * 1e-9;
    return rc;
}

void pir_server_destroy(pir_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    for (Slot& s : srv->slots) {
        if (s.d_block) cudaFreeAsync(s.d_block, s.stream);
        if (s.d_out) cudaFreeAsync(s.d_out, s.stream);
        if (s.stream) cudaStreamSynchronize(s.stream);
        cudaFreeHost(s.h_block);
        cudaFreeHost(s.h_out);
        for (void* h : s.retired_host) cudaFreeHost(h);
        cudaFree(s.d_counter);
        cudaFree(s.d_status);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    delete srv;
}

}  // extern "C"
