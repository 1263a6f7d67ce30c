"""GB300-native DPF-PIR server library: Python binding of libpir (include/pir.h).

Every function below has the name of the C entry point it calls and does
argument marshalling only; all computation happens in libpir's CUDA kernels
(server side) or its C++ host code (client key generation and
reconstruction).  There is no fallback: if the library is missing, import
raises.

Tables and device buffers are PyTorch CUDA tensors (torch.int32 holding u32
bit patterns); host keys are `bytes`.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libpir.so")

PIR_OK = 0
PIR_STATUS_BAD_KEY = 1
PIR_STATUS_SMEM_LAYOUT = 2
ERRORS = {-1: "PIR_ERR_ARG", -2: "PIR_ERR_DOMAIN", -3: "PIR_ERR_KEY", -4: "PIR_ERR_NOMEM", -5: "PIR_ERR_CUDA",
          -6: "PIR_ERR_TIMEOUT", -7: "PIR_ERR_BUSY", -8: "PIR_ERR_UNSUPPORTED", -9: "PIR_ERR_CANCELLED"}


class PirError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code == -5 or code == -4:
            detail = f" [{_lib.pir_last_cuda_error().decode()}]"
        super().__init__(f"{what}: {ERRORS.get(code, code)}{detail}")


class pir_table(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_uint64), ("width", ctypes.c_uint32),
                ("stride", ctypes.c_uint64)]


class pir_server_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("device_memory_budget", ctypes.c_uint64), ("streams", ctypes.c_uint32),
                ("item_log2", ctypes.c_uint32)]


class pir_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("batched_queries", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("cancelled", ctypes.c_uint64), ("grows", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


PIR_STRATEGY_FUSED = 0
PIR_STRATEGY_EXPAND_SCAN = 1
PIR_STRATEGY_FUSED_STAGED = 2


class pir_work_item(ctypes.Structure):
    _fields_ = [("table", ctypes.c_uint32), ("group", ctypes.c_uint32), ("range_log2", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("range", ctypes.c_uint64), ("query", ctypes.c_uint32 * 8)]


class pir_plan(ctypes.Structure):
    _fields_ = [("group", ctypes.c_uint32), ("range_log2", ctypes.c_uint32), ("vec", ctypes.c_uint32),
                ("ctas", ctypes.c_uint32), ("strategy", ctypes.c_uint32), ("tail_log2", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libpir.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    u8p, u32p, vp = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "pir_key_bytes": (ctypes.c_size_t, [ctypes.c_uint32]),
        "pir_domain_bits": (ctypes.c_uint32, [ctypes.c_uint64]),
        "pir_keygen": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, u8p, u8p, u8p]),
        "pir_keygen_prf": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u8p,
                                          u8p, u8p]),
        "pir_keygen_batch": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_size_t, vp, vp, ctypes.c_uint32, u8p, u8p, u8p,
                                            ctypes.c_uint32]),
        "pir_pbr_keygen": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, vp, ctypes.c_size_t, ctypes.c_uint32, u8p,
                                          u8p, u8p, vp]),
        "pir_server_eval_pbr": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_uint64, u8p, u32p, u32p, vp]),
        "pir_hotfull_keygen": (ctypes.c_int, [ctypes.c_uint64, vp, ctypes.c_uint64, vp, ctypes.c_size_t,
                                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u8p, u8p, u8p, u8p,
                                              u8p, vp]),
        "pir_key_check": (ctypes.c_int, [u8p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint32)]),
        "pir_reconstruct": (ctypes.c_int, [u32p, u32p, ctypes.c_size_t, u32p]),
        "pir_server_eval": (ctypes.c_int, [ctypes.POINTER(pir_table), u8p, ctypes.c_size_t, u32p, vp]),
        "pir_server_eval_device": (ctypes.c_int, [ctypes.POINTER(pir_table), u8p, ctypes.c_size_t, u32p, u32p, vp]),
        "pir_server_eval_device_plan": (ctypes.c_int, [ctypes.POINTER(pir_table), u8p, ctypes.c_size_t, u32p, u32p,
                                                       ctypes.POINTER(pir_plan), vp]),
        "pir_server_eval_range": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_uint64, ctypes.c_uint64, u8p,
                                                 ctypes.c_size_t, u32p, u32p, vp]),
        "pir_server_eval_noalloc": (ctypes.c_int, [ctypes.POINTER(pir_table), u8p, ctypes.c_size_t, u32p, vp]),
        "pir_expand_materialise": (ctypes.c_int, [ctypes.c_uint64, u8p, ctypes.c_size_t, u32p, ctypes.c_uint64, u32p,
                                                  vp]),
        "pir_contract_u32": (ctypes.c_int, [u32p, ctypes.c_uint64, ctypes.c_size_t, ctypes.POINTER(pir_table), u32p,
                                            ctypes.c_int, vp]),
        "pir_multi_plan_create": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_size_t, vp, ctypes.c_size_t,
                                                 ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
        "pir_multi_plan_destroy": (None, [vp]),
        "pir_multi_plan_inspect": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_size_t, vp, ctypes.c_size_t,
                                                  ctypes.c_uint32, vp, ctypes.c_size_t,
                                                  ctypes.POINTER(ctypes.c_uint64)]),
        "pir_multi_plan_layout": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(ctypes.c_uint64),
                                                 ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "pir_server_eval_multi": (ctypes.c_int, [vp, u8p, u32p, u32p, vp]),
        "pir_server_eval_multi_host": (ctypes.c_int, [vp, u8p, u32p, vp]),
        "pir_multi_graph_create": (ctypes.c_int, [vp, u8p, u32p, u32p, ctypes.POINTER(ctypes.c_void_p)]),
        "pir_graph_launch": (ctypes.c_int, [vp, vp]),
        "pir_graph_destroy": (None, [vp]),
        "pir_multi_autotune": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_size_t, vp, ctypes.c_size_t, u8p,
                                              u32p, vp, ctypes.POINTER(ctypes.c_uint32),
                                              ctypes.POINTER(ctypes.c_float)]),
        "pir_server_create": (ctypes.c_int, [ctypes.POINTER(pir_server_config), ctypes.POINTER(ctypes.c_void_p)]),
        "pir_server_register_table": (ctypes.c_int, [vp, ctypes.POINTER(pir_table), ctypes.POINTER(ctypes.c_uint32)]),
        "pir_submit": (ctypes.c_int, [vp, ctypes.c_uint32, u8p, u32p, ctypes.POINTER(ctypes.c_uint64)]),
        "pir_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]),
        "pir_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "pir_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, vp]),
        "pir_server_drain": (ctypes.c_int, [vp, ctypes.c_uint32]),
        "pir_server_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(pir_server_stats)]),
        "pir_server_replay": (ctypes.c_int, [vp, vp, vp, u8p, vp, ctypes.c_size_t, u32p, vp, vp,
                                             ctypes.POINTER(ctypes.c_double)]),
        "pir_server_destroy": (None, [vp]),
        "pir_autotune": (ctypes.c_int, [ctypes.POINTER(pir_table), u8p, ctypes.c_size_t, u32p, vp,
                                        ctypes.POINTER(pir_plan), ctypes.POINTER(ctypes.c_float)]),
        "pir_plan_for": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.POINTER(pir_plan)]),
        "pir_plan_pin": (ctypes.c_int, [ctypes.POINTER(pir_table), ctypes.c_size_t, ctypes.POINTER(pir_plan)]),
        "pir_plan_inspect": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_uint32,
                                            ctypes.POINTER(pir_plan)]),
        "pir_device_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]),
        "pir_staging_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "pir_error_string": (ctypes.c_char_p, [ctypes.c_int]),
        "pir_last_cuda_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH


def _check(rc: int, what: str):
    if rc != PIR_OK:
        raise PirError(rc, what)


def _buf(b: bytes):
    return ctypes.cast(ctypes.c_char_p(b), ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def table_of(t, rows: int | None = None) -> pir_table:
    """pir_table describing a 2-D CUDA tensor of 32-bit words; a pir_table is
    returned as it is (a caller may build the descriptor once and pass it to
    every call, as the C API's callers do)."""
    if isinstance(t, pir_table):
        return t
    assert t.dim() == 2 and t.element_size() == 4 and t.is_cuda and t.stride(1) == 1
    return pir_table(t.data_ptr(), t.shape[0] if rows is None else rows, t.shape[1], t.stride(0))


# ------------------------------------------------------------------ keys (host)

def pir_key_bytes(n: int) -> int:
    return int(_lib.pir_key_bytes(n))


def pir_domain_bits(rows: int) -> int:
    return int(_lib.pir_domain_bits(rows))


PIR_PRF_AES128, PIR_PRF_CHACHA20 = 0, 1


def pir_keygen(n: int, alpha: int, beta: int = 1, seed: bytes | None = None):
    return pir_keygen_prf(n, alpha, beta, PIR_PRF_AES128, seed)


def pir_keygen_prf(n: int, alpha: int, beta: int = 1, prf: int = PIR_PRF_AES128, seed: bytes | None = None):
    kb = pir_key_bytes(n)
    k0 = ctypes.create_string_buffer(kb)
    k1 = ctypes.create_string_buffer(kb)
    if seed is not None and len(seed) != 32:
        raise ValueError("seed must be 32 bytes")
    sp = _buf(seed) if seed is not None else None
    _check(_lib.pir_keygen_prf(n, alpha, beta & 0xFFFFFFFF, prf, sp, ctypes.cast(k0, ctypes.c_void_p),
                               ctypes.cast(k1, ctypes.c_void_p)), "pir_keygen_prf")
    return k0.raw, k1.raw


def pir_keygen_batch(n: int, alphas, betas=None, prf: int = PIR_PRF_AES128, seed: bytes | None = None,
                     threads: int = 0):
    """count key pairs at once; returns (keys0, keys1) as bytes, keys back to back."""
    import numpy as np

    a = np.ascontiguousarray(alphas, dtype=np.uint64)
    b = None if betas is None else np.ascontiguousarray(np.asarray(betas, dtype=np.uint64) & 0xFFFFFFFF,
                                                        dtype=np.uint32)
    if seed is not None and len(seed) != 32:
        raise ValueError("seed must be 32 bytes")
    kb = pir_key_bytes(n) * a.size
    k0 = ctypes.create_string_buffer(max(1, kb))
    k1 = ctypes.create_string_buffer(max(1, kb))
    _check(_lib.pir_keygen_batch(n, a.size, a.ctypes.data, b.ctypes.data if b is not None else None, prf,
                                 _buf(seed) if seed is not None else None, ctypes.cast(k0, ctypes.c_void_p),
                                 ctypes.cast(k1, ctypes.c_void_p), threads), "pir_keygen_batch")
    return k0.raw[:kb], k1.raw[:kb]


def pir_pbr_keygen(rows: int, bin_rows: int, indices, prf: int = PIR_PRF_AES128, seed: bytes | None = None):
    """Partial batch retrieval, client side: one key pair per bin.  Returns
    (keys0, keys1, kept) with kept[i] true when indices[i] is retrieved."""
    import numpy as np

    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    nbins = (rows + bin_rows - 1) // bin_rows if bin_rows else 0
    kb = pir_key_bytes(pir_domain_bits(bin_rows)) * nbins if bin_rows >= 2 else 0
    k0 = ctypes.create_string_buffer(max(1, kb))
    k1 = ctypes.create_string_buffer(max(1, kb))
    kept = np.zeros(max(1, idx.size), dtype=np.uint8)
    if seed is not None and len(seed) != 32:
        raise ValueError("seed must be 32 bytes")
    _check(_lib.pir_pbr_keygen(rows, bin_rows, idx.ctypes.data if idx.size else None, idx.size, prf,
                               _buf(seed) if seed is not None else None, ctypes.cast(k0, ctypes.c_void_p),
                               ctypes.cast(k1, ctypes.c_void_p), kept.ctypes.data), "pir_pbr_keygen")
    return k0.raw[:kb], k1.raw[:kb], kept[:idx.size].astype(bool)


def pir_hotfull_keygen(full_rows: int, hot_rows, indices, q_hot: int, q_full: int, prf: int = PIR_PRF_AES128,
                       seed: bytes | None = None):
    """Hot/full table split, client side: exactly q_hot hot-table and q_full
    full-table key pairs.  Returns (hot_keys0, hot_keys1, full_keys0,
    full_keys1, slot) with slot[i] the query that carries indices[i] (hot
    queries first), or -1 when it was dropped."""
    import numpy as np

    hot = np.ascontiguousarray(hot_rows, dtype=np.uint64)
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    hkb = pir_key_bytes(pir_domain_bits(hot.size)) * q_hot if hot.size >= 2 else 0
    fkb = pir_key_bytes(pir_domain_bits(full_rows)) * q_full if full_rows >= 2 else 0
    bufs = [ctypes.create_string_buffer(max(1, b)) for b in (hkb, hkb, fkb, fkb)]
    slot = np.zeros(max(1, idx.size), dtype=np.int64)
    if seed is not None and len(seed) != 32:
        raise ValueError("seed must be 32 bytes")
    _check(_lib.pir_hotfull_keygen(full_rows, hot.ctypes.data, hot.size, idx.ctypes.data if idx.size else None,
                                   idx.size, q_hot, q_full, prf, _buf(seed) if seed is not None else None,
                                   *[ctypes.cast(b, ctypes.c_void_p) for b in bufs], slot.ctypes.data),
           "pir_hotfull_keygen")
    return (bufs[0].raw[:hkb], bufs[1].raw[:hkb], bufs[2].raw[:fkb], bufs[3].raw[:fkb], slot[:idx.size].copy())


def pir_key_check(key: bytes):
    n = ctypes.c_uint32()
    party = ctypes.c_uint32()
    _check(_lib.pir_key_check(_buf(key), len(key), ctypes.byref(n), ctypes.byref(party)), "pir_key_check")
    return n.value, party.value


def pir_reconstruct(s0, s1):
    """(s0 + s1) mod 2^32 for host uint32 numpy arrays."""
    import numpy as np

    s0 = np.ascontiguousarray(s0, dtype=np.uint32)
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    out = np.empty_like(s0)
    _check(_lib.pir_reconstruct(s0.ctypes.data, s1.ctypes.data, s0.size, out.ctypes.data), "pir_reconstruct")
    return out


# ------------------------------------------------------------------ server

def _host_ptr(x):
    if isinstance(x, (bytes, bytearray)):
        return _buf(bytes(x))
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def pir_server_eval(table, keys, batch: int, out, stream=None):
    """Host keys (bytes, numpy or pinned CPU tensor holding batch * key_bytes
    back to back) -> `out` (host numpy/CPU tensor or CUDA tensor) of
    batch x width words."""
    tb = table_of(table)
    kbuf = bytes(keys) if isinstance(keys, (bytes, bytearray)) else keys
    kptr = _buf(kbuf) if isinstance(kbuf, bytes) else _host_ptr(kbuf)
    _check(_lib.pir_server_eval(ctypes.byref(tb), kptr, batch, _host_ptr(out), _stream(stream)), "pir_server_eval")
    return out


def pir_server_eval_noalloc(table, keys, batch: int, out, stream=None):
    """pir_server_eval through the library's fixed device staging region (no
    device allocation); host keys in, host `out` (numpy/CPU tensor) out."""
    tb = table_of(table)
    kbuf = bytes(keys) if isinstance(keys, (bytes, bytearray)) else keys
    kptr = _buf(kbuf) if isinstance(kbuf, bytes) else _host_ptr(kbuf)
    _check(_lib.pir_server_eval_noalloc(ctypes.byref(tb), kptr, batch, _host_ptr(out), _stream(stream)),
           "pir_server_eval_noalloc")
    return out


def pir_server_eval_device(table, dkeys, batch: int, dout, dstatus=None, stream=None):
    tb = table_of(table)
    _check(_lib.pir_server_eval_device(ctypes.byref(tb), dkeys.data_ptr(), batch, dout.data_ptr(),
                                       dstatus.data_ptr() if dstatus is not None else None, _stream(stream)),
           "pir_server_eval_device")
    return dout


def pir_server_eval_device_plan(table, dkeys, batch: int, dout, plan: pir_plan, dstatus=None, stream=None):
    tb = table_of(table)
    _check(_lib.pir_server_eval_device_plan(ctypes.byref(tb), dkeys.data_ptr(), batch, dout.data_ptr(),
                                            dstatus.data_ptr() if dstatus is not None else None,
                                            ctypes.byref(plan), _stream(stream)), "pir_server_eval_device_plan")
    return dout


def pir_server_eval_range(shard, row_lo: int, domain_rows: int, dkeys, batch: int, dout, dstatus=None, stream=None):
    tb = table_of(shard)
    _check(_lib.pir_server_eval_range(ctypes.byref(tb), row_lo, domain_rows, dkeys.data_ptr(), batch, dout.data_ptr(),
                                      dstatus.data_ptr() if dstatus is not None else None, _stream(stream)),
           "pir_server_eval_range")
    return dout


PIR_CONTRACT_IMAD = 0
PIR_CONTRACT_MMA_U8 = 1
PIR_CONTRACT_SCAN = 2
PIR_CONTRACT_TC_F16 = 3
PIR_CONTRACT_AUTO = 4
PIR_FAULT_WAIT_TIMEOUT = 1


def pir_server_eval_pbr(table, bin_rows: int, dkeys, dout, dstatus=None, stream=None):
    """Partial batch retrieval, server side: dout[b] = bin b's share (device)."""
    tb = table_of(table)
    _check(_lib.pir_server_eval_pbr(ctypes.byref(tb), bin_rows, dkeys.data_ptr(), dout.data_ptr(),
                                    dstatus.data_ptr() if dstatus is not None else None, _stream(stream)),
           "pir_server_eval_pbr")
    return dout


def pir_expand_materialise(rows: int, dkeys, batch: int, dshares, dstatus=None, stream=None):
    """Full share vectors into dshares (CUDA tensor [batch][ld], ld >= rows)."""
    assert dshares.dim() == 2 and dshares.stride(1) == 1 and dshares.shape[1] >= rows
    _check(_lib.pir_expand_materialise(rows, dkeys.data_ptr(), batch, dshares.data_ptr(), dshares.stride(0),
                                       dstatus.data_ptr() if dstatus is not None else None, _stream(stream)),
           "pir_expand_materialise")
    return dshares


def pir_contract_u32(dshares, batch: int, table, dout, engine: int = PIR_CONTRACT_IMAD, stream=None):
    tb = table_of(table)
    _check(_lib.pir_contract_u32(dshares.data_ptr(), dshares.stride(0), batch, ctypes.byref(tb), dout.data_ptr(),
                                 engine, _stream(stream)), "pir_contract_u32")
    return dout


def pir_selftest_bounded_wait(polls: int = 1 << 12, stream=None) -> int:
    """Runs the bounded-wait diagnostic; returns the library's code
    (PIR_ERR_TIMEOUT, -6, when the wait ran out as designed)."""
    return _lib.pir_selftest_bounded_wait(polls, _stream(stream))


def pir_device_status(clear: bool = False) -> int:
    """Library-wide device fault bits of the current device (PIR_FAULT_*)."""
    flags = ctypes.c_uint32(0)
    _check(_lib.pir_device_status(ctypes.byref(flags), int(clear)), "pir_device_status")
    return flags.value


def pir_staging_stats():
    """(reserved, used) bytes of the library's staging pool on the current device."""
    reserved, used = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.pir_staging_stats(ctypes.byref(reserved), ctypes.byref(used)), "pir_staging_stats")
    return int(reserved.value), int(used.value)


def pir_multi_plan_inspect(tables, table_of_key, item_log2: int = 0):
    """The planner's work items for these tables and queries, on the host.
    `tables` are (rows, width) pairs or (rows, width, stride, aligned) tuples
    (no memory is touched: data pointers are fake, 16-byte aligned when
    `aligned`).  Returns a list of dicts (table, group, range_log2, range,
    queries)."""
    import numpy as np

    descs = []
    for t in tables:
        rows, width = t[0], t[1]
        stride = t[2] if len(t) > 2 else width
        aligned = t[3] if len(t) > 3 else True
        descs.append(pir_table(4096 if aligned else 4100, rows, width, stride))
    arr = (pir_table * len(descs))(*descs)
    tok = np.ascontiguousarray(table_of_key, dtype=np.uint32)
    n = ctypes.c_uint64()
    _check(_lib.pir_multi_plan_inspect(arr, len(descs), tok.ctypes.data, tok.size, item_log2, None, 0,
                                       ctypes.byref(n)), "pir_multi_plan_inspect")
    items = (pir_work_item * max(1, n.value))()
    _check(_lib.pir_multi_plan_inspect(arr, len(descs), tok.ctypes.data, tok.size, item_log2, items, n.value,
                                       ctypes.byref(n)), "pir_multi_plan_inspect")
    return [{"table": w.table, "group": w.group, "range_log2": w.range_log2, "range": w.range,
             "queries": [q for q in w.query[:w.group] if q != 0xFFFFFFFF]} for w in items[:n.value]]


def _tables_array(tables):
    arr = (pir_table * len(tables))(*[table_of(t) for t in tables])
    return arr


class MultiPlan:
    """Owner of a pir_multi_plan (see include/pir.h); `layout` holds the key
    byte offsets, share word offsets and totals of the batch."""

    def __init__(self, tables, table_of_key, item_log2: int = 0):
        import numpy as np

        self._tables = _tables_array(tables)
        self.table_of_key = np.ascontiguousarray(table_of_key, dtype=np.uint32)
        self.batch = int(self.table_of_key.size)
        h = ctypes.c_void_p()
        _check(_lib.pir_multi_plan_create(self._tables, len(tables), self.table_of_key.ctypes.data, self.batch,
                                          item_log2, ctypes.byref(h)), "pir_multi_plan_create")
        self.handle = h
        self.key_offsets = np.zeros(self.batch, np.uint64)
        self.out_offsets = np.zeros(self.batch, np.uint64)
        kt, ot, it = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.pir_multi_plan_layout(h, self.key_offsets.ctypes.data, self.out_offsets.ctypes.data,
                                          ctypes.byref(kt), ctypes.byref(ot), ctypes.byref(it)),
               "pir_multi_plan_layout")
        self.key_bytes_total, self.out_words_total, self.items = kt.value, ot.value, it.value

    def close(self):
        if self.handle:
            _lib.pir_multi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pir_multi_plan_create(tables, table_of_key, item_log2: int = 0) -> MultiPlan:
    return MultiPlan(tables, table_of_key, item_log2)


def pir_server_eval_multi(plan: MultiPlan, dkeys, dout, dstatus=None, stream=None):
    _check(_lib.pir_server_eval_multi(plan.handle, dkeys.data_ptr(), dout.data_ptr(),
                                      dstatus.data_ptr() if dstatus is not None else None, _stream(stream)),
           "pir_server_eval_multi")
    return dout


def pir_server_eval_multi_host(plan: MultiPlan, keys, out, stream=None):
    """Host keys (plan layout; bytes, numpy or pinned tensor) -> host shares."""
    kbuf = bytes(keys) if isinstance(keys, (bytes, bytearray)) else keys
    kptr = _buf(kbuf) if isinstance(kbuf, bytes) else _host_ptr(kbuf)
    _check(_lib.pir_server_eval_multi_host(plan.handle, kptr, _host_ptr(out), _stream(stream)),
           "pir_server_eval_multi_host")
    return out


class Graph:
    def __init__(self, plan: MultiPlan, dkeys, dout, dstatus=None):
        h = ctypes.c_void_p()
        _check(_lib.pir_multi_graph_create(plan.handle, dkeys.data_ptr(), dout.data_ptr(),
                                           dstatus.data_ptr() if dstatus is not None else None, ctypes.byref(h)),
               "pir_multi_graph_create")
        self.handle = h
        self._keep = (plan, dkeys, dout, dstatus)

    def launch(self, stream=None):
        _check(_lib.pir_graph_launch(self.handle, _stream(stream)), "pir_graph_launch")

    def close(self):
        if self.handle:
            _lib.pir_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pir_multi_graph_create(plan: MultiPlan, dkeys, dout, dstatus=None) -> Graph:
    return Graph(plan, dkeys, dout, dstatus)


def pir_multi_autotune(tables, table_of_key, dkeys, dout, stream=None):
    """Returns (best item_log2, ms per launch) measured on the given batch."""
    import numpy as np

    tk = np.ascontiguousarray(table_of_key, dtype=np.uint32)
    arr = _tables_array(tables)
    best, ms = ctypes.c_uint32(), ctypes.c_float()
    _check(_lib.pir_multi_autotune(arr, len(tables), tk.ctypes.data, tk.size, dkeys.data_ptr(), dout.data_ptr(),
                                   _stream(stream), ctypes.byref(best), ctypes.byref(ms)), "pir_multi_autotune")
    return best.value, ms.value


class Server:
    """Owner of a pir_server (continuous batching over resident tables)."""

    def __init__(self, max_batch=0, max_inflight=0, device_memory_budget=0, streams=0, item_log2=0):
        cfg = pir_server_config(max_batch, max_inflight, device_memory_budget, streams, item_log2)
        h = ctypes.c_void_p()
        _check(_lib.pir_server_create(ctypes.byref(cfg), ctypes.byref(h)), "pir_server_create")
        self.handle = h
        self._tables = []

    def register_table(self, table) -> int:
        tid = ctypes.c_uint32()
        _check(_lib.pir_server_register_table(self.handle, ctypes.byref(table_of(table)), ctypes.byref(tid)),
               "pir_server_register_table")
        self._tables.append(table)
        return tid.value

    def submit(self, table_id: int, key: bytes, out) -> int:
        """`out`: host numpy uint32 array of the table's width (kept alive by the caller)."""
        t = ctypes.c_uint64()
        _check(_lib.pir_submit(self.handle, table_id, _buf(key), out.ctypes.data, ctypes.byref(t)), "pir_submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending, else the latency in ns."""
        lat = ctypes.c_int64()
        rc = _lib.pir_poll(self.handle, ticket, ctypes.byref(lat))
        if rc == -7:
            return None
        _check(rc, "pir_poll")
        return lat.value

    def cancel(self, ticket: int) -> bool:
        """True when the request was withdrawn before it ran; False when it is
        already running or done (poll it as usual)."""
        rc = _lib.pir_cancel(self.handle, ticket)
        if rc == -7:
            return False
        _check(rc, "pir_cancel")
        return True

    def drain(self, timeout_ms: int = 60000):
        _check(_lib.pir_server_drain(self.handle, timeout_ms), "pir_server_drain")

    def stats(self) -> dict:
        st = pir_server_stats()
        _check(_lib.pir_server_stats_get(self.handle, ctypes.byref(st)), "pir_server_stats_get")
        return st.as_dict()

    def replay(self, arrival_s, table_ids, keys: bytes, key_offsets, outs, out_offsets):
        """Open-loop replay; returns (latencies_ns array, elapsed seconds)."""
        import numpy as np

        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        tids = np.ascontiguousarray(table_ids, dtype=np.uint32)
        koff = np.ascontiguousarray(key_offsets, dtype=np.uint64)
        ooff = np.ascontiguousarray(out_offsets, dtype=np.uint64)
        lat = np.zeros(arr.size, np.int64)
        el = ctypes.c_double()
        _check(_lib.pir_server_replay(self.handle, arr.ctypes.data, tids.ctypes.data, _buf(keys), koff.ctypes.data,
                                      arr.size, outs.ctypes.data, ooff.ctypes.data, lat.ctypes.data,
                                      ctypes.byref(el)), "pir_server_replay")
        return lat, el.value

    def close(self):
        if self.handle:
            _lib.pir_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pir_server_create(**cfg) -> Server:
    return Server(**cfg)


def pir_plan_pin(table, batch: int, plan=None):
    """Pins `plan` (a pir_plan) for this table shape and batch size, as if the
    autotuner had chosen it; None removes the entry (the heuristic answers)."""
    _check(_lib.pir_plan_pin(ctypes.byref(table_of(table)), batch, ctypes.byref(plan) if plan is not None else None),
           "pir_plan_pin")


def pir_autotune(table, dkeys, batch: int, dout, stream=None):
    """Times launch shapes on this batch; returns (pir_plan, ms per launch).
    The library keeps using the winner for this table shape and batch size."""
    plan, ms = pir_plan(), ctypes.c_float()
    _check(_lib.pir_autotune(ctypes.byref(table_of(table)), dkeys.data_ptr(), batch, dout.data_ptr(),
                             _stream(stream), ctypes.byref(plan), ctypes.byref(ms)), "pir_autotune")
    return plan, ms.value


def pir_plan_for(rows: int, width: int, batch: int) -> pir_plan:
    p = pir_plan()
    _check(_lib.pir_plan_for(rows, width, batch, ctypes.byref(p)), "pir_plan_for")
    return p


def pir_plan_inspect(rows: int, width: int, batch: int, sms: int) -> pir_plan:
    """The heuristic plan for a device with `sms` SMs, on the host only."""
    p = pir_plan()
    _check(_lib.pir_plan_inspect(rows, width, batch, sms, ctypes.byref(p)), "pir_plan_inspect")
    return p


def pir_error_string(code: int) -> str:
    return _lib.pir_error_string(code).decode()
