// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "pir.h"

#include <nvtx3/nvToolsExt.h>

namespace pir {

// ---- host AES-128 (aes_host.cpp) -------------------------------------------
// FIPS-197 AES-128 on 32-bit columns (byte r of column c at bits 8r of word c).
struct Aes128 {
    uint32_t rk[44];
    void set_key(const uint8_t key[16]);
    void encrypt(const uint8_t in[16], uint8_t out[16]) const;
};
const uint8_t* aes_sbox();  // the 256-byte S-box, derived once from GF(2^8)

// ---- key layout -------------------------------------------------------------
constexpr uint32_t kKeyMagic = 0x4B465044u;  // "DPFK" little-endian
constexpr uint32_t kKeyVersion = 1;
inline size_t key_bytes(uint32_t n) { return PIR_KEY_HEADER_BYTES + 64u * (size_t)n; }
inline size_t codeword_offset(uint32_t d, uint32_t t, uint32_t b) {
    return PIR_KEY_HEADER_BYTES + 64u * (size_t)(d - 1) + 32u * t + 16u * b;
}

// ---- device launch (dpf_eval.cu) --------------------------------------------
struct EvalRequest {
    const uint32_t* table;  // row `row_lo` of the evaluated rows
    uint64_t row_lo, row_hi;
    uint32_t width;
    uint64_t stride;
    uint32_t n;
    const uint8_t* dkeys;
    uint32_t batch;
    uint32_t* dout;       // batch x width, accumulated into (zeroed by the caller)
    uint32_t* dstatus;    // optional
};

// ---- multi-table work list (multi.cpp builds it, dpf_eval.cu runs it) --------
constexpr uint32_t kNoQuery = 0xffffffffu;
struct MultiTable {  // device copy of one registered table
    const uint32_t* data;
    uint64_t rows;
    uint64_t stride;
    uint32_t width;
    uint32_t n;
    uint32_t key_bytes;
    uint32_t range_log2;  // rows per item of this table: 2^range_log2
};
struct MultiItem {  // (table, row range, up to 8 queries of that table)
    uint32_t table;
    uint32_t group;  // query slots of the item: 1, 2, 4 or 8 (the queries in q[0..group))
    uint64_t range;  // first row = range << range_log2
    uint32_t q[8];   // query indices, kNoQuery for empty slots
};
struct MultiParams {
    const MultiTable* tables;
    const MultiItem* items;
    uint64_t nitems;
    const uint64_t* key_off;  // byte offset of key q in keys
    const uint64_t* out_off;  // word offset of share q in out
    const uint8_t* keys;
    uint32_t* out;
    uint32_t* status;
    uint64_t* counter;  // next item; zeroed before each launch
};
int launch_multi(const MultiParams& mp, bool vec, void* stream);

// Host side of the multi-table planner (multi.cpp): fills `mt` from the
// descriptors and appends the work items; offsets of keys (bytes) and shares
// (words) in query order.  Returns PIR_OK or an error code.
struct MultiLayout {
    std::vector<MultiTable> tables;
    std::vector<MultiItem> items;
    std::vector<uint64_t> key_off, out_off;
    uint64_t key_total = 0, out_total = 0;
    bool vec = true;
    bool auto_range = false;  // rows per item chosen per table from its queries (item_log2 == 0)
};
int describe_tables(const pir_table* tables, size_t ntables, uint32_t item_log2, MultiLayout& lay);
int plan_items(const uint32_t* table_of_key, size_t batch, MultiLayout& lay);
int multi_group();          // queries per item
int multi_max_range_log2(); // largest rows-per-item exponent the kernel supports
// rows per item (log2) from the fused planner's cost model for one table of
// `rows` rows with nqg groups of `group` query slots
int plan_range_log2(uint64_t rows, uint32_t n, uint32_t group, uint32_t nqg);
// consumer threads of a fused work item (a compile-time tuning knob shared with
// the kernels): they cover a row in W / VEC column chunks, one chunk each at most
#ifndef PIR_CONSUMER_WARPS
#define PIR_CONSUMER_WARPS 8
#endif
constexpr uint32_t kFusedConsumerThreads = 32u * PIR_CONSUMER_WARPS;

int device_sm_count();
// The same for a device with `sms` SMs (host only).
int plan_fused_sms(uint64_t rows_evaluated, uint64_t row_lo, uint32_t n, uint32_t width, uint32_t batch, bool vec_ok,
                   int sms, pir_plan* plan);
int plan_fused(uint64_t rows_evaluated, uint64_t row_lo, uint32_t n, uint32_t width, uint32_t batch, bool vec_ok,
               pir_plan* plan);
int plan_check(const pir_plan& plan, uint32_t n, uint32_t width, bool vec_ok);
// The same for PIR_STRATEGY_FUSED_STAGED, which also needs the table's row
// pitch (words) and leaves room for its shared-memory ring.
int plan_check_staged(const pir_plan& plan, uint32_t n, uint32_t width, uint64_t stride, bool vec_ok);
// Pieces per cut item of the last, partial round (log2) for a plan's shape.
uint32_t plan_tail_log2(uint64_t row_lo, uint64_t rows, uint32_t n, uint32_t group, uint32_t batch,
                        uint32_t range_log2);
int launch_fused(const EvalRequest& req, const pir_plan& plan, void* stream);
// partial batch retrieval: req.batch bins of bin_rows rows, req.row_hi = table rows
int plan_bins(uint64_t bin_rows, uint32_t n, uint32_t width, uint32_t nbins, pir_plan* plan);
int launch_bins(const EvalRequest& req, uint64_t bin_rows, const pir_plan& plan, void* stream);
int launch_materialise(const EvalRequest& req, const pir_plan& plan, uint32_t* shares, uint64_t ld, void* stream);
// partial batch retrieval in one launch: the bins' trees breadth first, then each
// CTA's own rows of a dense table (clears dout); PIR_ERR_UNSUPPORTED outside its layouts
int launch_pbr_fused(const uint32_t* table, uint64_t rows, uint32_t width, uint64_t stride, uint64_t bin_rows,
                     uint32_t n, const uint8_t* dkeys, uint32_t nbins, uint32_t* dout, uint32_t* dstatus,
                     void* stream);

// share matrix x table mod 2^32 (contract.cu); out is accumulated into
int launch_contract(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                    uint32_t width, uint64_t rows, uint32_t* out, int engine, void* stream);

// the same product on the tcgen05 tensor cores with fp16 limbs (contract_tc.cu)
int launch_contract_tc(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                       uint32_t width, uint64_t rows, uint32_t* out, void* stream);

// streaming scan engine for a few queries (scan.cu): eight queries per pass
bool scan_supported(const uint32_t* shares, uint64_t ld, const uint32_t* table, uint64_t stride, uint32_t width);
int launch_scan(const uint32_t* shares, uint64_t ld, uint32_t batch, const uint32_t* table, uint64_t stride,
                uint32_t width, uint64_t rows, uint32_t* out, void* stream);
// the diagonal form (partial batch retrieval): shares[k] belongs to row k and to
// query k / bin_rows; out[b] = sum over bin b's rows (bin_rows a multiple of the
// engine's chunk, which scan_bins_supported checks)
bool scan_bins_supported(const uint32_t* table, uint64_t stride, uint32_t width, uint64_t bin_rows);
int launch_scan_bins(const uint32_t* shares, const uint32_t* table, uint64_t stride, uint32_t width, uint64_t rows,
                     uint64_t bin_rows, uint32_t* out, void* stream);
// dst[i] = src[i] for i < words by a kernel (scan.cu): either side may be
// pinned host memory mapped into the device's address space
int launch_words_copy(const uint32_t* src, uint32_t* dst, uint64_t words, void* stream);
// diagnostic: a bounded wait that must run out (scan.cu)
int selftest_bounded_wait(uint32_t polls, void* stream);
// library-wide device fault bits (PIR_FAULT_*), read on the current device
int device_faults(uint32_t* flags, bool clear);
// device address of that fault word on the current device (nullptr on a CUDA error)
uint32_t* device_fault_word();

// A named range of the calling host thread for timeline tools (Nsight Systems
// and the like); without a tool attached the push and pop do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// error bookkeeping (api.cpp)
int cuda_fail(int cuda_error_code, const char* what);

}  // namespace pir
