"""CPU oracle for DPF-PIR over Z_2^32 — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never imports the product.

The arithmetic lives in ``dpf_oracle.c`` (plain C, compiled here with gcc):
AES-128 from FIPS-197 (S-box derived from its GF(2^8) definition), the DPF
recurrence of Eqs. p1-p3 of the paper (Sec. 3.1), BGI16 key generation in the
paper's codeword form, and the server's inner product T x Eval(k, .) mod 2^32.
This module is argument marshalling only.

Every function here is pinned by ``tests/test_oracle_*.py``; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

KEY_HEADER_BYTES = 32


def build(force: bool = False) -> str:
    """Compile dpf_oracle.c into _build/liboracle.so (portable C, no ISA flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_sbox.argtypes = [u8p]
        lib.orc_gf_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
        lib.orc_gf_mul.restype = ctypes.c_uint8
        lib.orc_aes128_key_expansion.argtypes = [u8p, u8p]
        lib.orc_aes128_encrypt.argtypes = [u8p, u8p, u8p]
        lib.orc_prf.argtypes = [u8p, ctypes.c_uint8, u8p]
        lib.orc_key_bytes.argtypes = [ctypes.c_uint32]
        lib.orc_key_bytes.restype = ctypes.c_size_t
        lib.orc_gen.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, u8p, u8p, u8p, u8p, u8p]
        lib.orc_gen.restype = ctypes.c_int
        lib.orc_gen_prf.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, u8p, u8p, u8p,
                                    u8p, u8p]
        lib.orc_gen_prf.restype = ctypes.c_int
        lib.orc_chacha20_block.argtypes = [u8p, ctypes.c_uint32, u8p, u8p]
        lib.orc_chacha_quarter_round.argtypes = [u32p, u32p, u32p, u32p]
        lib.orc_prf_id.argtypes = [ctypes.c_int, u8p, ctypes.c_uint8, u8p]
        lib.orc_eval.argtypes = [u8p, ctypes.c_uint64, u32p]
        lib.orc_eval.restype = ctypes.c_int
        lib.orc_full_eval.argtypes = [u8p, ctypes.c_uint64, u32p]
        lib.orc_full_eval.restype = ctypes.c_int
        lib.orc_answer_range.argtypes = [u8p, u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64, u32p]
        lib.orc_answer_range.restype = ctypes.c_int
        lib.orc_reconstruct.argtypes = [u32p, u32p, ctypes.c_size_t, u32p]
        lib.orc_node.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint64, u8p]
        lib.orc_node.restype = ctypes.c_int
        lib.orc_key_parse.argtypes = [u8p, u32p, u32p, u32p]
        lib.orc_key_parse.restype = ctypes.c_int
        _lib = lib
        return lib


def _u8(buf):
    arr = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8)) if not isinstance(buf, np.ndarray) else buf
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u32(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------- AES / PRF

def sbox() -> bytes:
    out = np.zeros(256, np.uint8)
    _load().orc_sbox(_u8(out)[1])
    return out.tobytes()


def gf_mul(a: int, b: int) -> int:
    return int(_load().orc_gf_mul(a, b))


def aes128_key_expansion(key: bytes) -> bytes:
    """FIPS-197 Sec. 5.2: the 44 words w[0..43], 176 bytes."""
    k, kp = _u8(key)
    out = np.zeros(176, np.uint8)
    _load().orc_aes128_key_expansion(kp, _u8(out)[1])
    return out.tobytes()


def aes128_encrypt(key: bytes, block: bytes) -> bytes:
    k, kp = _u8(key)
    b, bp = _u8(block)
    out = np.zeros(16, np.uint8)
    _load().orc_aes128_encrypt(kp, bp, _u8(out)[1])
    return out.tobytes()


def prf(seed: bytes, x: int, prf_id: int = 0) -> bytes:
    """PRF_seed(x): prf_id 0 = AES-128, 1 = ChaCha20 (see dpf_oracle.c)."""
    s, sp = _u8(seed)
    out = np.zeros(16, np.uint8)
    _load().orc_prf_id(prf_id, sp, x, _u8(out)[1])
    return out.tobytes()


PRF_AES128, PRF_CHACHA20 = 0, 1


def chacha20_block(key: bytes, counter: int, nonce: bytes) -> bytes:
    """RFC 8439 Sec. 2.3 block function: 64 bytes."""
    k, kp = _u8(key)
    nn, np_ = _u8(nonce)
    out = np.zeros(64, np.uint8)
    _load().orc_chacha20_block(kp, counter, np_, _u8(out)[1])
    return out.tobytes()


def chacha_quarter_round(a: int, b: int, c: int, d: int):
    v = [ctypes.c_uint32(x) for x in (a, b, c, d)]
    _load().orc_chacha_quarter_round(*[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


# ---------------------------------------------------------------- DPF

def key_bytes(n: int) -> int:
    return int(_load().orc_key_bytes(n))


def gen(n: int, alpha: int, beta: int, seed0: bytes, seed1: bytes, rand_c0: bytes, prf_id: int = 0):
    """Gen with explicit randomness: two 16-byte roots and n*2*16 codeword bytes."""
    if len(seed0) != 16 or len(seed1) != 16 or len(rand_c0) != 32 * n:
        raise ValueError("gen randomness has the wrong size")
    kb = key_bytes(n)
    k0 = np.zeros(kb, np.uint8)
    k1 = np.zeros(kb, np.uint8)
    s0, s0p = _u8(seed0)
    s1, s1p = _u8(seed1)
    rc, rcp = _u8(rand_c0)
    _check(_load().orc_gen_prf(n, alpha, beta & 0xFFFFFFFF, prf_id, s0p, s1p, rcp, _u8(k0)[1], _u8(k1)[1]), "gen")
    return k0.tobytes(), k1.tobytes()


def key_parse(key: bytes):
    k, kp = _u8(key)
    n = ctypes.c_uint32()
    party = ctypes.c_uint32()
    cw = ctypes.c_uint32()
    _check(_load().orc_key_parse(kp, ctypes.byref(n), ctypes.byref(party), ctypes.byref(cw)), "key_parse")
    return n.value, party.value, cw.value


def eval_point(key: bytes, j: int) -> int:
    """Eval(k, j) by the root-to-leaf path (branch form)."""
    k, kp = _u8(key)
    y = ctypes.c_uint32()
    _check(_load().orc_eval(kp, j, ctypes.byref(y)), "eval")
    return y.value


def full_eval(key: bytes, L: int) -> np.ndarray:
    """Eval(k, j) for all j < L, computed level by level."""
    k, kp = _u8(key)
    y = np.zeros(L, np.uint32)
    _check(_load().orc_full_eval(kp, L, _u32(y)), "full_eval")
    return y


def answer(key: bytes, table: np.ndarray, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Server share: sum_{lo<=j<hi} Eval(k, j) * T[j] mod 2^32 (table holds all L rows)."""
    table = np.ascontiguousarray(table, dtype=np.uint32)
    L, W = table.shape
    hi = L if hi is None else hi
    k, kp = _u8(key)
    out = np.zeros(W, np.uint32)
    sub = table[lo:hi] if hi > lo else table[:1]
    sub = np.ascontiguousarray(sub)
    _check(_load().orc_answer_range(kp, _u32(sub), L, W, W, lo, hi, _u32(out)), "answer")
    return out


def contract(S: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Share matrix x table mod 2^32: out[b][w] = sum_k S[b][k] T[k][w]
    (Sec. 3.1, the batched product).  numpy's integer matmul on uint64 is the
    step: products of u32 fit in 64 bits and the wrap mod 2^64 preserves the
    residue mod 2^32."""
    S = np.ascontiguousarray(S, dtype=np.uint32).astype(np.uint64)
    T = np.ascontiguousarray(T, dtype=np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        return ((S @ T) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def pbr_plan(rows: int, bin_rows: int, indices):
    """Partial batch retrieval, client side (Sec. 4, batch PIR): the table is
    cut into ceil(rows / bin_rows) bins of bin_rows rows and every bin gets one
    query.  A bin yields one entry: the first wanted index that falls in it is
    retrieved, any later one in the same bin is dropped.  A bin nobody wants
    gets a dummy query (alpha 0, beta 0).  Returns (alphas, betas, kept)."""
    nbins = -(-rows // bin_rows)
    alphas, betas, kept = [0] * nbins, [0] * nbins, []
    for idx in indices:
        b = int(idx) // bin_rows
        if betas[b] == 0:
            alphas[b], betas[b] = int(idx) - b * bin_rows, 1
            kept.append(True)
        else:
            kept.append(False)
    return alphas, betas, kept


def pbr_answer(keys, table: np.ndarray, bin_rows: int) -> np.ndarray:
    """Partial batch retrieval, server side: bin b's share is the answer of
    key b over the bin's own rows, table[b * bin_rows : (b + 1) * bin_rows]."""
    table = np.ascontiguousarray(table, dtype=np.uint32)
    return np.stack([answer(k, table[b * bin_rows:(b + 1) * bin_rows]) for b, k in enumerate(keys)])


def hotfull_plan(full_rows: int, hot_rows, indices, q_hot: int, q_full: int):
    """Frequency-based hot/full split, client side (Sec. 4): exactly q_hot
    queries to the hot table (hot row h = full row hot_rows[h]) and q_full to
    the full table per request.  A wanted hot row uses a hot query while any
    remain; other rows, and hot rows past the hot budget, use full queries
    while any remain; the rest are dropped.  Unused queries are dummies
    (alpha 0, beta 0).  Returns (hot_alphas, hot_betas, full_alphas,
    full_betas, slots); slots[i] = s (hot query s), q_hot + s (full query s)
    or -1 (dropped)."""
    where = {int(r): h for h, r in enumerate(hot_rows)}
    ha, hb, fa, fb, slots = [0] * q_hot, [0] * q_hot, [0] * q_full, [0] * q_full, []
    nh = nf = 0
    for idx in indices:
        idx = int(idx)
        if idx in where and nh < q_hot:
            ha[nh], hb[nh] = where[idx], 1
            slots.append(nh)
            nh += 1
        elif nf < q_full:
            fa[nf], fb[nf] = idx, 1
            slots.append(q_hot + nf)
            nf += 1
        else:
            slots.append(-1)
    return ha, hb, fa, fb, slots


def reconstruct(s0: np.ndarray, s1: np.ndarray) -> np.ndarray:
    s0 = np.ascontiguousarray(s0, dtype=np.uint32)
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    out = np.zeros_like(s0)
    _load().orc_reconstruct(_u32(s0), _u32(s1), s0.size, _u32(out))
    return out


def node(key: bytes, d: int, j: int) -> bytes:
    """The tree node P(d, j) (16 bytes) of the key's expansion."""
    k, kp = _u8(key)
    out = np.zeros(16, np.uint8)
    _check(_load().orc_node(kp, d, j, _u8(out)[1]), "node")
    return out.tobytes()
