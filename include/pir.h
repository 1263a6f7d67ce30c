/*
 * pir.h — C ABI of the GB300 DPF-PIR server library (libpir).
 *
 * Two-server private information retrieval over an embedding table T with L
 * rows of W uint32 words, after Lam et al., "GPU-based Private Information
 * Retrieval for On-Device Machine Learning Inference" (arXiv 2301.10904).
 *
 *   client: Gen(1^lambda, alpha) -> (k_0, k_1)            (Sec. 3.1, "DPF-PIR")
 *   server sigma: share_sigma = T x Eval(k_sigma, {0..L-1})  (Sec. 3.1, Eqs. p1-p3)
 *   client: T[alpha] * beta = share_0 + share_1 (mod 2^32)   (Sec. 3.1)
 *
 * All table, share and output arithmetic is integer mod 2^32; all tree
 * arithmetic is 128-bit XOR with AES-128 or ChaCha20 as the PRF (Sec. 3.2.6).
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device
 *    memory of the current device; "host" pointers are ordinary or pinned
 *    host memory.  `stream` is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).
 *  - The caller owns every buffer.  The library keeps no pointer after a
 *    call returns.
 *  - Return value: PIR_OK (0) or a negative PIR_ERR_* code.  No exceptions
 *    cross the ABI.  Device-side key errors are reported through an
 *    optional device status word (bit PIR_STATUS_BAD_KEY) because they are
 *    only seen once the kernel runs.
 *  - Calls that take device outputs are asynchronous on `stream`; calls that
 *    write host outputs synchronize `stream` before returning.
 *  - Domain: L >= 2 rows, n = ceil(log2 L) <= 40 tree levels; leaves j >= L
 *    of the 2^n-leaf tree are evaluated but never multiplied.
 *
 * Key wire format (32 + 64 n bytes, little-endian, 16-byte aligned fields):
 *   [0,4) "DPFK"  [4] version 1  [5] n  [6] party sigma (0/1)  [7] PRF id
 *   [8,12) cw_out (u32)  [12,16) 0  [16,32) root seed P(0,0) of this party
 *   [32 + 64(d-1) + 32t + 16b, +16) = codeword C_t[b][d], d = 1..n, t,b in {0,1}
 * The 64 n codeword bytes are the paper's key size (Table 4: 896 B at 16K
 * entries, 1280 B at 1M, 1408 B at 4M).
 */
#ifndef PIR_H
#define PIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------- */
#define PIR_OK 0
#define PIR_ERR_ARG (-1)         /* null pointer, zero size, bad shape or stride */
#define PIR_ERR_DOMAIN (-2)      /* key's n differs from ceil(log2 rows), alpha >= 2^n */
#define PIR_ERR_KEY (-3)         /* malformed key header, unknown party */
#define PIR_ERR_NOMEM (-4)       /* device or host allocation failed */
#define PIR_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define PIR_ERR_TIMEOUT (-6)     /* a bounded wait ran out */
#define PIR_ERR_BUSY (-7)        /* admission refused (serving) */
#define PIR_ERR_UNSUPPORTED (-8) /* shape outside the kernels' limits */
#define PIR_ERR_CANCELLED (-9)   /* the request was cancelled before it ran (serving) */

#define PIR_STATUS_BAD_KEY 1u    /* device status bit: some key failed validation */
#define PIR_STATUS_SMEM_LAYOUT 2u /* device status bit: a kernel found its shared memory at an
                                     unexpected window offset and did nothing (the host checks the
                                     device's reserved shared memory first, so this is a guard) */

#define PIR_KEY_HEADER_BYTES 32
#define PIR_MAX_DOMAIN_BITS 40

/* PRF of a key's tree (header byte 7).  AES-128: PRF_s(x) = AES-128_s of the
 * block (x, 0, ..., 0) (Sec. 3.1, Sec. 3.2.6).  ChaCha20 (Sec. 3.2.6,
 * Table 5): PRF_s(x) = bytes [16x, 16x+16) of ChaCha20 block 0 (RFC 8439)
 * under key s || 0^128 with an all-zero nonce.  Every server entry point
 * takes either, per key. */
#define PIR_PRF_AES128 0u
#define PIR_PRF_CHACHA20 1u

/* A table resident in device memory: row j of the table (j counted from the
 * first row `data` points at) starts at data + j * stride.  data must be
 * 4-byte aligned; 16-byte alignment with stride % 4 == 0 enables 128-bit
 * loads. */
typedef struct pir_table {
    const uint32_t* data; /* device */
    uint64_t rows;        /* L */
    uint32_t width;       /* W, words per entry */
    uint64_t stride;      /* words between consecutive rows, >= width */
} pir_table;

/* How a single-table evaluation runs: the fused kernel (expansion and product
 * in one launch, Sec. 3.2.4), or expansion into stream-ordered scratch followed
 * by the streaming table scan (Sec. 3.2.2's level-by-level strategy), or the
 * fused kernel with its table scan staged through shared memory: one more warp
 * has the bulk-copy engine move each hand-off's table rows into a ring of
 * shared-memory stages ahead of the consumers, so that a group of one to four
 * queries keeps enough of the table in flight (the share vector still never
 * leaves the SM).  PIR_STRATEGY_FUSED_STAGED needs 16-byte rows (vec 4), group
 * <= 4, stride <= 256 words and subtrees shallow enough to leave at least two
 * DFS stack levels free for the ring (range_log2 - min(log2(512/group),
 * range_log2 - 1) <= 7); otherwise PIR_ERR_UNSUPPORTED. */
#define PIR_STRATEGY_FUSED 0u
#define PIR_STRATEGY_EXPAND_SCAN 1u
#define PIR_STRATEGY_FUSED_STAGED 2u

/* Launch shape of the fused kernel.  `group` queries share one CTA and one
 * pass over each table tile; each work item covers 2^range_log2 consecutive
 * rows, and the grid (min(items, SMs) CTAs) takes items round-robin.  When
 * the items do not fill the last round, each item of that round is cut into
 * 2^tail_log2 pieces of 2^(range_log2 - tail_log2) rows, so that every CTA
 * takes part in it (0: no cut; the planner picks it by its cost model).
 * strategy PIR_STRATEGY_EXPAND_SCAN ignores group/range_log2/vec/tail_log2
 * (the expansion is planned on its own) and needs 16-byte rows with
 * stride <= 1024. */
typedef struct pir_plan {
    uint32_t group;      /* queries per CTA: 1, 2, 4 or 8 */
    uint32_t range_log2; /* log2 rows per work item, 1 <= range_log2 <= n */
    uint32_t vec;        /* table words per load: 4 (128-bit) or 1 */
    uint32_t ctas;       /* resulting grid size (output of pir_plan_for) */
    uint32_t strategy;   /* PIR_STRATEGY_FUSED, _EXPAND_SCAN or _FUSED_STAGED */
    uint32_t tail_log2;  /* 0..min(3, range_log2 - 1): pieces per item of a partial last round */
} pir_plan;

/* ---- keys (host only) ----------------------------------------------- */

/* Key size in bytes for an n-level tree: 32 + 64 n. */
size_t pir_key_bytes(uint32_t n);

/* Number of tree levels for a table of `rows` rows: ceil(log2 rows)
 * (1 for rows <= 2).  Returns 0 for rows == 0 or rows > 2^40. */
uint32_t pir_domain_bits(uint64_t rows);

/* Gen(1^128, alpha) of Sec. 3.1, with the correction-word construction of
 * BGI16 [dpf_1] (the paper defers key generation to it), in the codeword
 * form C_t[b][d] of Eq. p3.  Writes pir_key_bytes(n) bytes to each of key0
 * and key1 (host).  seed: 32 bytes of key material for a deterministic
 * AES-128-CTR generator (tests, reproducible benchmarks), or NULL to draw
 * from the operating system's entropy source.  Errors: PIR_ERR_ARG (null
 * keys, n == 0 or n > 40), PIR_ERR_DOMAIN (alpha >= 2^n). */
int pir_keygen(uint32_t n, uint64_t alpha, uint32_t beta, const uint8_t* seed, uint8_t* key0, uint8_t* key1);

/* pir_keygen with the tree's PRF chosen: PIR_PRF_AES128 (what pir_keygen
 * uses) or PIR_PRF_CHACHA20.  Errors as pir_keygen; PIR_ERR_ARG for an
 * unknown prf. */
int pir_keygen_prf(uint32_t n, uint64_t alpha, uint32_t beta, uint32_t prf, const uint8_t* seed, uint8_t* key0,
                   uint8_t* key1);

/* Many keys at once (the client's Gen for a batch of queries, Sec. 3.1):
 * key pair i is pir_keygen_prf(n, alphas[i], betas ? betas[i] : 1, prf,
 * seed_i), written at keys0/keys1 + i * pir_key_bytes(n) (host).  seed_i is
 * the i-th 32-byte block of the AES-128-CTR stream of `seed` (32 bytes, or
 * NULL: a master seed from the operating system's entropy source), so the
 * keys do not depend on `threads` (0 = one per hardware thread).  Errors: as
 * pir_keygen_prf, for the first failing key. */
int pir_keygen_batch(uint32_t n, size_t count, const uint64_t* alphas, const uint32_t* betas, uint32_t prf,
                     const uint8_t* seed, uint8_t* keys0, uint8_t* keys1, uint32_t threads);

/* Partial batch retrieval, client side (Sec. 4, batch PIR after [multihot]):
 * the table's `rows` rows are cut into nbins = ceil(rows / bin_rows) bins of
 * bin_rows rows (the last may be shorter) and one query goes to every bin,
 * a DPF over n_b = pir_domain_bits(bin_rows) levels.  Of the `count` wanted
 * row indices, the first that falls in a bin is retrieved (kept[i] = 1,
 * alpha = index - bin * bin_rows, beta = 1); a later one in the same bin is
 * dropped (kept[i] = 0; a bin yields one entry).  Bins with no wanted index
 * get a dummy query (alpha = 0, beta = 0), so neither server learns which bins
 * were wanted.  keys0/keys1: nbins * pir_key_bytes(n_b) bytes each (host),
 * generated as pir_keygen_batch with `seed`.  Errors: PIR_ERR_ARG (bin_rows <
 * 2, null buffers), PIR_ERR_DOMAIN (an index >= rows). */
int pir_pbr_keygen(uint64_t rows, uint64_t bin_rows, const uint64_t* indices, size_t count, uint32_t prf,
                   const uint8_t* seed, uint8_t* keys0, uint8_t* keys1, uint8_t* kept);

/* Frequency-based hot/full table split, client side (Sec. 4, "Frequency-Based
 * Hot Table Split"): next to the full table (full_rows rows) the server holds a
 * hot table of hot_count rows, hot row h being full-table row hot_rows[h]
 * (hot_rows strictly increasing; the client's copy of this map is the paper's
 * on-device index of hot entries).  Every request sends exactly q_hot queries
 * to the hot table and q_full to the full table, so neither server learns how
 * many wanted rows are hot or how many rows are wanted.  Wanted full-table
 * rows, in order: a hot row goes to the hot table while hot queries remain;
 * any other row, or a hot row once the hot queries are used, goes to the full
 * table while full queries remain; the rest are dropped (slot[i] = -1).
 * slot[i] = s for hot query s, q_hot + s for full query s.  Unused queries
 * are dummies (alpha 0, beta 0).  Keys: hot keys over
 * pir_domain_bits(hot_count) levels (q_hot key pairs back to back), full keys
 * over pir_domain_bits(full_rows) levels, each set generated as
 * pir_keygen_batch with a 32-byte seed drawn from `seed`'s AES-128-CTR stream
 * (first block pair: hot, second: full; NULL: operating-system entropy).
 * Errors: PIR_ERR_ARG, PIR_ERR_DOMAIN (a wanted row >= full_rows). */
int pir_hotfull_keygen(uint64_t full_rows, const uint64_t* hot_rows, uint64_t hot_count, const uint64_t* indices,
                       size_t count, uint32_t q_hot, uint32_t q_full, uint32_t prf, const uint8_t* seed,
                       uint8_t* hot_keys0, uint8_t* hot_keys1, uint8_t* full_keys0, uint8_t* full_keys1,
                       int64_t* slot);

/* Validates a key's header (magic, version, n, party, length == 32 + 64 n).
 * On success stores n and the party (0 or 1).  Errors: PIR_ERR_ARG,
 * PIR_ERR_KEY. */
int pir_key_check(const uint8_t* key, size_t len, uint32_t* n, uint32_t* party);

/* Client reconstruction (Sec. 3.1): out[i] = s0[i] + s1[i] mod 2^32 (host). */
int pir_reconstruct(const uint32_t* s0, const uint32_t* s1, size_t w, uint32_t* out);

/* ---- server evaluation ---------------------------------------------- */

/* share_sigma[q] = sum_{j<L} Eval(k_q, j) * T[j]  (mod 2^32) for each of the
 * `batch` keys (Sec. 3.1 "Eval"; fused with the table product as in
 * Sec. 3.2.4, so the L-long share vector never reaches device memory).
 * keys: host, batch * pir_key_bytes(n) bytes back to back, every key with
 * n == pir_domain_bits(t->rows).  out: batch x width words, host or device
 * (detected).  With a host `out` the call returns after the result is
 * there.  A small call with a host `out` (keys and shares up to 32 KiB
 * each) is staged in buffers of the calling thread (64 KiB of device and
 * 96 KiB of pinned host memory per thread and device, kept until the thread
 * exits) and runs as a CUDA graph built on the first call of its shape
 * (table, batch, launch plan; up to 8 kept per thread): the keys and a
 * zeroed share area reach the device in one copy, and the GPU runs that
 * copy, the kernels and the copy back without waiting for the host between
 * them.  Other calls stage keys (and host-bound shares) in stream-ordered
 * device memory from a pool the library creates per device, which keeps up
 * to 256 MiB of freed staging mapped between calls.  Errors: PIR_ERR_ARG,
 * PIR_ERR_KEY, PIR_ERR_DOMAIN, PIR_ERR_NOMEM, PIR_ERR_CUDA,
 * PIR_ERR_UNSUPPORTED, and, with a host `out`, PIR_ERR_TIMEOUT when a
 * bounded wait in this call's kernels gave up (the expand-and-scan and
 * staged strategies have such waits; the shares are then incomplete and
 * PIR_FAULT_WAIT_TIMEOUT stays set in the device status).  With a device
 * `out` the call is asynchronous: check pir_device_status after
 * synchronizing. */
int pir_server_eval(const pir_table* t, const uint8_t* keys, size_t batch, uint32_t* out, void* stream);

/* Same computation with keys and outputs already in device memory (the
 * steady-state serving form).  dkeys: device, batch * pir_key_bytes(n)
 * bytes, 16-byte aligned.  dout: device, batch x width words, overwritten.
 * dstatus: optional device word; PIR_STATUS_BAD_KEY is OR-ed into it when a
 * key fails validation on the device, and that query's share is 0.
 * Strategy: the autotuned one for this shape (pir_autotune), else the fused
 * kernel, except for one or two queries against a table of 128 MiB or more
 * whose rows hold at least 64 words per query, with 16-byte rows (stride <=
 * 1024): those are expanded into stream-ordered scratch of batch x rows x 4
 * bytes from the library's pool and contracted by the streaming scan
 * (PIR_STRATEGY_EXPAND_SCAN; faster there on GB300, where each table row read
 * serves too few queries for the fused kernel's product side).  Same result
 * bit for bit.  Asynchronous on `stream`; the expand-and-scan and staged
 * strategies' bounded waits report a wait that gave up only through
 * PIR_FAULT_WAIT_TIMEOUT (pir_device_status), which callers check after
 * synchronizing. */
int pir_server_eval_device(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout,
                           uint32_t* dstatus, void* stream);

/* As pir_server_eval_device with an explicit launch shape (autotuning,
 * sweeps).  plan->ctas is ignored.  Errors: PIR_ERR_UNSUPPORTED for a shape
 * the kernels cannot run. */
int pir_server_eval_device_plan(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout,
                                uint32_t* dstatus, const pir_plan* plan, void* stream);

/* Index-range evaluation, the unit of multi-GPU sharding (Sec. 3.2.7: each
 * GPU evaluates the DPF on a subset of indices and the partial results are
 * summed, the final reduction being linear).  Computes
 *   dout[q] = sum_{row_lo <= j < row_hi} Eval(k_q, j) * T[j]   (mod 2^32)
 * where `shard` holds rows row_lo..row_hi-1 (shard->data points at row
 * row_lo, shard->rows == row_hi - row_lo) and `domain_rows` is the full
 * table's L, which fixes n.  Asynchronous; dout overwritten. */
int pir_server_eval_range(const pir_table* shard, uint64_t row_lo, uint64_t domain_rows, const uint8_t* dkeys,
                          size_t batch, uint32_t* dout, uint32_t* dstatus, void* stream);

/* Allocation-free form of pir_server_eval for callers that cannot let a
 * library allocate device memory: a serving runtime that owns the whole
 * device-memory budget, or a request path that must not take the
 * allocator's locks or risk the device synchronisation an allocation can
 * cause.  The paper has no counterpart; this is a deployment variant.
 * Same inputs, output and result as pir_server_eval with host keys and a
 * host `out` (batch x width words): keys and shares are staged through one
 * fixed 256 KiB region of device memory that belongs to the library image
 * (192 KiB for keys, 64 KiB for shares), so batch * pir_key_bytes(n) must
 * be <= 196608 and batch * width * 4 <= 65536, else PIR_ERR_UNSUPPORTED.
 * The call calls no device allocator and returns after `out` holds the
 * shares.  The first call on a device looks up the region's device address
 * (one-time set-up; repeated once if the device's primary context has been
 * replaced, e.g. after cudaDeviceReset); make that first call before any
 * stream capture.  All calls share the region, which keeps the last call's
 * contents (the share area is cleared at the start of each call): calls that
 * overlap on the GPU race, so issue them from one stream and one thread at a
 * time.  `out` must be host memory (PIR_ERR_ARG for device or managed
 * memory).  Errors: as pir_server_eval, plus PIR_ERR_UNSUPPORTED for the size
 * limit. */
int pir_server_eval_noalloc(const pir_table* t, const uint8_t* keys, size_t batch, uint32_t* out, void* stream);

/* ---- many tables in one launch ------------------------------------- */

/* Opaque launch plan for one batch of queries spread over several resident
 * tables of uneven sizes and widths (batched execution, Sec. 3.2.1, across
 * tables).  Holds a device-resident work list: items of (table, row range of
 * 2^r rows, up to 8 queries of that table), r = min(ceil(log2 rows),
 * item_log2), or with item_log2 = 0 chosen per table for its queries.  Keys and shares of the batch are laid out back to back in
 * query order; pir_multi_plan_layout reports the offsets. */
typedef struct pir_multi_plan pir_multi_plan;

/* tables: host array of `ntables` descriptors (device data, every width
 * <= 512 words); table_of_key: host array, table index of each of the
 * `batch` queries; item_log2: rows per work item as a power of two (at most
 * 15), or 0 to let the planner choose per table: a cost model of dependent
 * tree levels against work per item, given the table's query count (a lone
 * query on a large table gets up to 2^18-row items).  The tables must stay resident
 * while the plan is used.  Allocates device memory for the work list (the
 * plan owns it).  Errors: PIR_ERR_ARG, PIR_ERR_DOMAIN, PIR_ERR_UNSUPPORTED
 * (width), PIR_ERR_NOMEM, PIR_ERR_CUDA. */
int pir_multi_plan_create(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                          uint32_t item_log2, pir_multi_plan** plan);

void pir_multi_plan_destroy(pir_multi_plan* plan);

/* One work item of a multi-table plan, as the planner lays it out. */
typedef struct pir_work_item {
    uint32_t table;      /* table index */
    uint32_t group;      /* query slots: 1, 2, 4 or 8 */
    uint32_t range_log2; /* the table's rows per item, log2 */
    uint32_t pad;
    uint64_t range;      /* first row = range << range_log2 */
    uint32_t query[8];   /* query indices (query[s] for s < group; 0xffffffff for an empty slot) */
} pir_work_item;

/* The work items pir_multi_plan_create would build for these arguments,
 * computed on the host only (no device memory, no device needed; with no
 * device visible the planner assumes one SM).  *nitems gets the count; if
 * items is non-NULL, up to `capacity` items are written.  Errors as
 * pir_multi_plan_create, without the device ones. */
int pir_multi_plan_inspect(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                           uint32_t item_log2, pir_work_item* items, size_t capacity, uint64_t* nitems);

/* Layout of a plan's batch (all outputs optional, host): key_offsets[q]
 * (bytes) and out_offsets[q] (u32 words) for q < batch, the key buffer's
 * total bytes, the share buffer's total words, the number of work items. */
int pir_multi_plan_layout(const pir_multi_plan* plan, uint64_t* key_offsets, uint64_t* out_offsets,
                          uint64_t* key_bytes_total, uint64_t* out_words_total, uint64_t* items);

/* One persistent launch over the whole work list: for every query q,
 * dout[out_offsets[q] .. + width of its table) = its share (Sec. 3.1, fused
 * as in Sec. 3.2.4).  dkeys: device, 16-byte aligned, key q at
 * key_offsets[q] with n = ceil(log2 rows) of its table.  dout (device) is
 * overwritten; dstatus as for pir_server_eval_device.  Asynchronous and
 * capturable in a CUDA graph (a memset of dout, a memset of the plan's item
 * counter, one kernel).  One plan serves one stream at a time: concurrent
 * launches of the same plan race on its item counter. */
int pir_server_eval_multi(const pir_multi_plan* plan, const uint8_t* dkeys, uint32_t* dout, uint32_t* dstatus,
                          void* stream);

/* pir_server_eval_multi from host buffers: copies `keys` (host, the plan's
 * key layout) to device staging owned by the plan (allocated on the first
 * call), launches, and copies the shares to `out` (host, the plan's share
 * layout); returns after `out` is filled. */
int pir_server_eval_multi_host(pir_multi_plan* plan, const uint8_t* keys, uint32_t* out, void* stream);

/* A CUDA graph holding pir_server_eval_multi for fixed buffers: replaying it
 * evaluates whatever keys dkeys holds at launch time. */
typedef struct pir_graph pir_graph;
int pir_multi_graph_create(const pir_multi_plan* plan, const uint8_t* dkeys, uint32_t* dout, uint32_t* dstatus,
                           pir_graph** graph);
int pir_graph_launch(pir_graph* graph, void* stream);
void pir_graph_destroy(pir_graph* graph);

/* Autotuner: times pir_server_eval_multi for item_log2 = 15, 14, ..., 11 on
 * the given batch (device keys and a device share buffer of the plan's
 * layout; synchronizes `stream`) and returns the fastest in *best_item_log2
 * (and its time per launch in *best_ms when non-null). */
int pir_multi_autotune(const pir_table* tables, size_t ntables, const uint32_t* table_of_key, size_t batch,
                       const uint8_t* dkeys, uint32_t* dout, void* stream, uint32_t* best_item_log2, float* best_ms);

/* ---- serving loop ---------------------------------------------------- */

/* A server with resident tables that batches queries as they arrive
 * (continuous cross-table batching).  The paper tunes a batch size per table
 * offline (Sec. 3.2.1; Sec. 5 tunes it per experiment);
 * here the batch is whatever arrived while the previous batch ran.
 * Requests are admitted into max_inflight slots (from a device-memory
 * budget); a full pool refuses with PIR_ERR_BUSY.  A worker thread packs
 * each batch's keys and work list into one pinned block and issues copy-in,
 * the multi-table kernel and copy-out on one of `streams` CUDA streams, so a
 * new batch overlaps the running one.  Results go straight into the
 * caller's host buffer; latency runs from arrival to that copy. */
typedef struct pir_server pir_server;

typedef struct pir_server_config {
    uint32_t max_batch;            /* queries per launch; 0 = 2048 */
    uint32_t max_inflight;         /* admitted but unfinished queries; 0 = derived from the budget */
    uint64_t device_memory_budget; /* bytes of key, share and work-list space behind max_inflight; 0 = 256 MiB */
    uint32_t streams;              /* batches in flight at once, 1..8; 0 = 2 */
    uint32_t item_log2;            /* rows per work item as a power of two; 0 = per table per batch (see pir_multi_plan_create) */
} pir_server_config;

typedef struct pir_server_stats {
    uint64_t submitted, completed, rejected, batches, batched_queries;
    uint32_t max_inflight;
    uint64_t cancelled;
    uint64_t grows; /* batch buffers reallocated because a batch outgrew them (sized for max_batch at start) */
} pir_server_stats;

/* Starts the worker thread on the current device.  cfg may be NULL. */
int pir_server_create(const pir_server_config* cfg, pir_server** server);

/* Registers a resident table (device data, width <= 512 words); the server
 * keeps the descriptor, the caller keeps the memory alive until destroy. */
int pir_server_register_table(pir_server* server, const pir_table* t, uint32_t* table_id);

/* Admits one query: key (host, pir_key_bytes(n) bytes, n of the table; copied
 * before return) for table_id; its share (width words) is written to `out`
 * (host) when done.  *ticket identifies it for pir_poll.  Errors:
 * PIR_ERR_BUSY (pool full: retry later), PIR_ERR_KEY, PIR_ERR_DOMAIN,
 * PIR_ERR_ARG. */
int pir_submit(pir_server* server, uint32_t table_id, const uint8_t* key, uint32_t* out, uint64_t* ticket);

/* PIR_OK when the ticket's share is in its buffer (the ticket is then
 * released; *latency_ns = arrival to completion), PIR_ERR_BUSY while it is
 * queued or running, PIR_ERR_ARG for an unknown ticket, or the error that
 * failed its batch. */
int pir_poll(pir_server* server, uint64_t ticket, int64_t* latency_ns);

/* Waits until nothing is queued or running; PIR_ERR_TIMEOUT after timeout_ms. */
int pir_server_drain(pir_server* server, uint32_t timeout_ms);

int pir_server_stats_get(pir_server* server, pir_server_stats* stats);

/* Open-loop load replay (measurement tool): submits query i at arrival_s[i]
 * seconds after the call starts (a full pool delays the submission, and the
 * latency still counts from the scheduled arrival), with keys at
 * keys + key_offsets[i] and shares to outs + out_offsets[i] (host), then
 * drains.  latency_ns[i] receives each latency; *elapsed_s the wall time. */
int pir_server_replay(pir_server* server, const double* arrival_s, const uint32_t* table_ids, const uint8_t* keys,
                      const uint64_t* key_offsets, size_t count, uint32_t* outs, const uint64_t* out_offsets,
                      int64_t* latency_ns, double* elapsed_s);

/* Withdraws a submitted request that has not been batched yet: its ticket is
 * released and its output buffer is not written.  Returns PIR_OK when it was
 * cancelled, PIR_ERR_BUSY when it is already running or done (poll it as
 * usual), PIR_ERR_ARG for an unknown ticket. */
int pir_cancel(pir_server* server, uint64_t ticket);

/* Drains, stops the worker and frees the server's buffers. */
void pir_server_destroy(pir_server* server);

/* ---- partial batch retrieval, server side ---------------------------- */

/* Sec. 4 (batch PIR, after [multihot]): key b is a DPF over bin b of the
 * table, rows [b * bin_rows, min((b + 1) * bin_rows, t->rows)), and
 *   dout[b][w] = sum_{j < rows of bin b} Eval(k_b, j) * T[b * bin_rows + j][w]   (mod 2^32)
 * for b < nbins = ceil(t->rows / bin_rows).  Strategy: when bin_rows is a
 * multiple of the streaming scan's chunk (e.g. powers of two >= 256 rows at
 * 16-64-word rows), every bin's share vector is expanded into stream-ordered
 * scratch (nbins x bin_rows x 4 bytes from the library's pool) and the table
 * is streamed once, each chunk of rows multiplying its own bin's shares;
 * otherwise one fused launch in which every CTA work item holds up to 8 bins
 * side by side, each with its own rows.  Same result bit for bit.  dkeys: device, nbins *
 * pir_key_bytes(pir_domain_bits(bin_rows)) bytes, 16-byte aligned (as
 * written by pir_pbr_keygen).  dout: device, nbins x width, overwritten.
 * dstatus: as pir_server_eval_device.  Needs bin_rows >= 2, 16-byte aligned
 * rows (t->data 16-byte aligned; stride and width multiples of 4) and width
 * <= 1024, else PIR_ERR_ARG / PIR_ERR_UNSUPPORTED.  Asynchronous. */
int pir_server_eval_pbr(const pir_table* t, uint64_t bin_rows, const uint8_t* dkeys, uint32_t* dout,
                        uint32_t* dstatus, void* stream);

/* ---- materialised (unfused) baseline ------------------------------- */

#define PIR_CONTRACT_IMAD 0   /* CUDA-core 32-bit multiply-add */
#define PIR_CONTRACT_MMA_U8 1 /* tensor-core u8 x u8 -> s32 MMAs on 8-bit limbs (10 per u32 product), exact */
#define PIR_CONTRACT_SCAN 2   /* streaming table scan for a few queries, bound by HBM bandwidth */
#define PIR_CONTRACT_TC_F16 3 /* tcgen05 tensor cores, fp16 signed 8-bit limbs, fp32 TMEM accumulators, exact */
#define PIR_CONTRACT_AUTO 4   /* the engine measured fastest for the shape (see pir_contract_u32) */

/* Expansion only (the level-by-level strategy's output, Sec. 3.2.2): writes
 * the full share vectors dshares[q * ld + j] = Eval(k_q, j) for j < rows,
 * q < batch (device, u32; ld >= rows; 16-byte aligned with ld % 4 == 0
 * enables vector stores).  O(batch x rows) device memory, which the fused
 * path avoids (Sec. 3.2.4).  Keys as for pir_server_eval_device; a key that
 * fails validation gets an all-zero share vector and sets PIR_STATUS_BAD_KEY
 * in *dstatus.  Asynchronous. */
int pir_expand_materialise(uint64_t rows, const uint8_t* dkeys, size_t batch, uint32_t* dshares, uint64_t ld,
                           uint32_t* dstatus, void* stream);

/* dout[q][w] = sum_{j < t->rows} dshares[q * ld + j] * T[j][w]  (mod 2^32),
 * the share-matrix x table product of Sec. 3.1 (a batch of queries as one
 * matrix-matrix product).  engine (same result bit for bit):
 *  - PIR_CONTRACT_IMAD: 64 x 64 output tiles on CUDA cores, any batch;
 *  - PIR_CONTRACT_MMA_U8: the same tiles on the tensor pipe (8-bit limbs);
 *  - PIR_CONTRACT_TC_F16: 128-query x 64-word tiles (32 words when
 *    t->width <= 32) on the fifth-generation tensor cores (tcgen05.mma
 *    with accumulators in tensor memory): every u32 is split into four
 *    signed 8-bit limbs held exactly in fp16, the ten limb products of
 *    the low 32 bits accumulate exactly in fp32 for 256 values of k at a
 *    time and are then folded into u32 totals.  With dshares and t->data
 *    16-byte aligned and ld and t->stride multiples of 4 the raw tiles
 *    arrive by tensor-map copies (PIR_TC_TENSOR_MAPS=0 in the environment
 *    selects the kernel that loads them itself, as for other operands; the
 *    result is the same).  One CTA per SM (up to 222 KB of shared memory)
 *    holding its SM's tensor memory (512 columns; 256 for 32-word tiles)
 *    while it runs, so a kernel that uses tensor memory on the same SM at
 *    the same time waits for it.  Its
 *    waits are bounded like the scan's; one that gives up sets
 *    PIR_FAULT_WAIT_TIMEOUT, and then the whole launch's dout is invalid,
 *    not only that CTA's tile: the CTA frees its tensor memory after a
 *    last bounded wait for its own MMAs, which may still be writing there
 *    when the next CTA on that SM allocates it;
 *  - PIR_CONTRACT_SCAN: for a few queries, where the product is bound by
 *    reading the table (Sec. 3.2.4): the copy engine streams table rows and
 *    share words through shared memory, eight queries per pass over the
 *    table.  Needs dshares and t->data 16-byte aligned, ld, t->stride and
 *    t->width multiples of 4 and t->stride <= 1024, else
 *    PIR_ERR_UNSUPPORTED.  Its waits on the copies are bounded: one that
 *    gives up leaves dout incomplete and sets PIR_FAULT_WAIT_TIMEOUT (see
 *    pir_device_status);
 *  - PIR_CONTRACT_AUTO: the fastest of these as measured on GB300 for the
 *    shape: the streaming scan for at most 16 queries (32 when t->width <=
 *    32) where its layout conditions hold, the tcgen05 engine otherwise
 *    (IMAD and the u8-limb MMAs are slower than one of the two at every
 *    batch).
 * dout (device, batch x width) is overwritten.  Asynchronous. */
int pir_contract_u32(const uint32_t* dshares, uint64_t ld, size_t batch, const pir_table* t, uint32_t* dout,
                     int engine, void* stream);

/* The launch shape the library picks for (rows, width, batch) on the current
 * device (heuristic, or the autotuned entry when one is cached). */
int pir_plan_for(uint64_t rows, uint32_t width, size_t batch, pir_plan* plan);

/* The heuristic launch shape for (rows, width, batch) on a device with `sms`
 * SMs (1..65536), computed on the host only (no device needed, no autotuned
 * entry consulted): what pir_plan_for answers untuned on such a device.
 * Errors: PIR_ERR_ARG, PIR_ERR_DOMAIN, PIR_ERR_UNSUPPORTED (width). */
int pir_plan_inspect(uint64_t rows, uint32_t width, size_t batch, uint32_t sms, pir_plan* plan);

/* Pins `plan` for evaluations of this table shape and batch: stores it where
 * pir_autotune stores its winner, for (current device, t->rows, t->width,
 * batch rounded up to a power of two, whether 128-bit loads apply), after
 * the checks of an explicit plan (pir_server_eval_device_plan).  Restores a
 * plan measured in an earlier process, or fixes one for a deployment.  A NULL
 * `plan` removes the entry, so that the heuristic answers again.  Host only
 * (no launch).  Errors: PIR_ERR_ARG, PIR_ERR_DOMAIN, PIR_ERR_UNSUPPORTED
 * (a plan outside the kernels' limits for this table). */
int pir_plan_pin(const pir_table* t, size_t batch, const pir_plan* plan);

/* Autotuner of the single-table strategy and launch shape (the paper tunes
 * batch and strategy per table size, Sec. 3.2.1 and 3.2.5): times, on this
 * table and batch (device keys dkeys, device shares dout; synchronizes
 * `stream`), the fused kernel for query groups G in {8,4,2,1} and rows per
 * item 2^r around the heuristic's choice, the staged fused kernel
 * (PIR_STRATEGY_FUSED_STAGED) for G <= 4 at the heuristic's rows per item and
 * half of it, and, where the layout allows it and batch <= 8, the
 * expand-and-scan strategy; remembers the fastest for
 * (device, rows, width, batch rounded up to a power of two).
 * pir_server_eval, pir_server_eval_device and pir_plan_for use it from then
 * on (pir_server_eval_noalloc always runs the fused kernel on its own plan).  Returns it in *plan and its time per launch in
 * *best_ms (optional). */
int pir_autotune(const pir_table* t, const uint8_t* dkeys, size_t batch, uint32_t* dout, void* stream,
                 pir_plan* plan, float* best_ms);

/* Library-wide device fault bits, set by a kernel whose bounded wait gave
 * up (the kernel then returns early; its output is incomplete, and for the
 * tcgen05 contraction every output of that launch is invalid).  The bits
 * stay set until cleared, so the outputs of every asynchronous call since
 * they were last clear are suspect.  Reads the bits of the current device
 * (synchronous) and clears them if `clear`. */
#define PIR_FAULT_WAIT_TIMEOUT 1u
int pir_device_status(uint32_t* flags, int clear);

/* Device memory of the library's staging pool on the current device (the
 * stream-ordered pool the host-buffer entry points stage keys, shares and
 * expand-and-scan scratch in): bytes it holds from the driver and bytes in
 * use by allocations not yet freed.  Creates the pool (no memory) if the
 * device has none yet.  Errors: PIR_ERR_ARG, PIR_ERR_CUDA. */
int pir_staging_stats(uint64_t* reserved_bytes, uint64_t* used_bytes);

/* Diagnostic of the bounded waits on the current device: runs a one-thread
 * kernel that waits on an mbarrier nothing ever completes, for at most
 * `polls` try_wait polls, so that the bound runs out as a stuck copy's would.
 * The kernel sets PIR_FAULT_WAIT_TIMEOUT in the device status and returns;
 * the context stays usable.  Synchronizes `stream`.  Returns PIR_ERR_TIMEOUT
 * when the wait ran out as designed, PIR_OK if it did not (it cannot), or a
 * CUDA error. */
int pir_selftest_bounded_wait(uint32_t polls, void* stream);

/* Human-readable name of an error code (static string). */
const char* pir_error_string(int code);

/* Text of the last CUDA error seen by this thread (static per thread). */
const char* pir_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PIR_H */
