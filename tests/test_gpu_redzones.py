"""Out-of-bounds checks on the GPU without a memory checker.  Every device
entry point runs on operands placed inside larger allocations whose guard
bands, before and after, hold seeded random words.  Tables are also given rows
padded past their width with random words.  A write out of bounds changes a
guard band or a padding word.  A read out of bounds pulls those random words
into a result, which then differs from the oracle's.  After each call the
results are compared with the oracle, every read-only operand (table, keys,
shares) with its initial contents word for word, and every output's guard
bands likewise."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import make_keys

pytestmark = pytest.mark.gpu
GUARD = 4096  # words on each side: 16 KiB, so every payload stays 16-byte aligned


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import oracle
    import paper_2301_10904_gb300 as pir

    return torch, pir, oracle


class Guarded:
    """n 32-bit words in one device allocation between two guard bands of
    seeded random words; the payload starts as `init` (random words if None)."""

    def __init__(self, torch, n, seed, init=None, device="cuda"):
        g = np.random.Generator(np.random.PCG64(seed))
        host = g.integers(0, 1 << 32, GUARD + n + GUARD, dtype=np.uint64).astype(np.uint32)
        if init is not None:
            host[GUARD:GUARD + n] = np.asarray(init, dtype=np.uint32).reshape(-1)
        self.host, self.n = host, n
        self.dev = torch.from_numpy(host.view(np.int32).copy()).to(device)

    def words(self):
        return self.dev[GUARD:GUARD + self.n]

    def _now(self):
        return self.dev.cpu().numpy().view(np.uint32)

    def guards_intact(self):
        d = self._now()
        return (np.array_equal(d[:GUARD], self.host[:GUARD])
                and np.array_equal(d[GUARD + self.n:], self.host[GUARD + self.n:]))

    def unchanged(self):
        return np.array_equal(self._now(), self.host)


def guarded_table(torch, T, pad, seed, device="cuda"):
    """T (rows x W) stored in rows of W + pad words whose padding is random."""
    rows, W = T.shape
    stride = W + pad
    full = np.random.Generator(np.random.PCG64(seed + 1)).integers(0, 1 << 32, (rows, stride),
                                                                   dtype=np.uint64).astype(np.uint32)
    full[:, :W] = T
    buf = Guarded(torch, rows * stride, seed, full, device)
    return buf, buf.words().view(rows, stride)[:, :W]


def guarded_bytes(torch, raw, seed):
    """A byte string (keys) in a guarded allocation; returns the buffer and a
    uint8 view of exactly len(raw) bytes."""
    nwords = -(-len(raw) // 4)
    payload = np.frombuffer(raw + bytes(4 * nwords - len(raw)), dtype=np.uint32)
    buf = Guarded(torch, nwords, seed, payload)
    return buf, buf.words().view(torch.uint8)[:len(raw)]


def guarded_out(torch, rows, cols, seed):
    buf = Guarded(torch, rows * cols, seed)
    return buf, buf.words().view(rows, cols)


def intact(*bufs):
    return all(b.guards_intact() for b in bufs)


def _answers(orc, keys, T, lo=0, hi=None):
    return np.stack([orc.answer(k, T, lo, hi) for k in keys])


@pytest.mark.parametrize("strategy", [0, 1, 2], ids=["fused", "expand_scan", "fused_staged"])
@pytest.mark.parametrize("rows,W,B,pad", [(4096 + 77, 16, 3, 4), (1 << 14, 64, 8, 4), (1000, 3, 5, 1),
                                          (3000, 8, 9, 8), ((1 << 15) + 1000, 32, 2, 4), (2, 1, 1, 3),
                                          ((1 << 16) + 5, 64, 1, 4)])
def test_server_eval_redzones(env, rows, W, B, pad, strategy):
    torch, pir, orc = env
    if strategy == 1 and (W % 4 or pad % 4 or B > 8):
        pytest.skip("the expand-and-scan strategy needs 16-byte rows and at most 8 queries")
    if strategy == 2 and (W % 4 or pad % 4 or rows < 4):
        pytest.skip("the staged scan needs 16-byte rows")
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(rows + 3, rows, W)
    ks0, _ = make_keys(orc, n, wl.alphas(rows + 5, rows, B), [1] * B, rows + 7)
    tbuf, table = guarded_table(torch, T, pad, 101)
    kbuf, dkeys = guarded_bytes(torch, b"".join(ks0), 202)
    obuf, out = guarded_out(torch, B, W, 303)
    if strategy == 2:
        from test_gpu_staged import staged_plan

        plan = staged_plan(pir, rows, W, B)
    else:
        plan = pir.pir_plan_for(rows, W, B)
        plan.strategy = strategy
    pir.pir_server_eval_device_plan(table, dkeys, B, out, plan)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), _answers(orc, ks0, T))
    assert tbuf.unchanged() and kbuf.unchanged() and intact(obuf)
    assert pir.pir_device_status(clear=True) == 0


def test_range_shard_redzones(env):
    torch, pir, orc = env
    L, W, B, lo, hi = 5000, 16, 6, 1024, 3000
    n = pir.pir_domain_bits(L)
    T = wl.table_u32(17, L, W)
    ks0, _ = make_keys(orc, n, wl.alphas(18, L, B), [1] * B, 19)
    tbuf, shard = guarded_table(torch, T[lo:hi], 4, 111)
    kbuf, dkeys = guarded_bytes(torch, b"".join(ks0), 212)
    obuf, out = guarded_out(torch, B, W, 313)
    pir.pir_server_eval_range(shard, lo, L, dkeys, B, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), _answers(orc, ks0, T, lo, hi))
    assert tbuf.unchanged() and kbuf.unchanged() and intact(obuf)


@pytest.mark.parametrize("rows,bin_rows,W,pad", [(5000, 1024, 16, 4), (1 << 14, 256, 32, 4), (3000, 700, 8, 4)])
def test_pbr_redzones(env, rows, bin_rows, W, pad):
    torch, pir, orc = env
    T = wl.table_u32(rows + 1, rows, W)
    rng = np.random.Generator(np.random.PCG64(rows))
    alphas, betas, _ = orc.pbr_plan(rows, bin_rows, rng.integers(0, rows, rows // bin_rows).tolist())
    nb = (bin_rows - 1).bit_length()
    rnd = wl.key_randomness(rows + 2, nb, len(alphas))
    keys = [orc.gen(nb, a, b, r0, r1, c0)[0] for (r0, r1, c0), a, b in zip(rnd, alphas, betas)]
    tbuf, table = guarded_table(torch, T, pad, 121)
    kbuf, dkeys = guarded_bytes(torch, b"".join(keys), 222)
    obuf, out = guarded_out(torch, len(keys), W, 323)
    pir.pir_server_eval_pbr(table, bin_rows, dkeys, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.pbr_answer(keys, T, bin_rows))
    assert tbuf.unchanged() and kbuf.unchanged() and intact(obuf)


def test_multi_table_redzones(env):
    torch, pir, orc = env
    shapes, pads = [(1000, 16), (4096, 4), (1 << 13, 64), (3, 8)], [4, 8, 4, 1]
    assign = [0, 2, 2, 1, 3, 0, 2, 2, 1, 0, 2]
    Ts = [wl.table_u32(50 + i, r, w) for i, (r, w) in enumerate(shapes)]
    guarded = [guarded_table(torch, T, p, 130 + i) for i, (T, p) in enumerate(zip(Ts, pads))]
    ks0 = []
    for q, t in enumerate(assign):
        k0, _ = make_keys(orc, pir.pir_domain_bits(shapes[t][0]), [wl.alphas(q + 60, shapes[t][0], 1)[0]], [1],
                          q + 70)
        ks0.append(k0[0])
    plan = pir.pir_multi_plan_create([v for _, v in guarded], assign)
    raw = bytearray(plan.key_bytes_total)
    for q, k in enumerate(ks0):
        o = int(plan.key_offsets[q])
        raw[o:o + len(k)] = k
    kbuf, dkeys = guarded_bytes(torch, bytes(raw), 232)
    obuf, out = guarded_out(torch, 1, plan.out_words_total, 333)
    pir.pir_server_eval_multi(plan, dkeys, out.view(-1))
    torch.cuda.synchronize()
    flat = out.view(-1).cpu().numpy().view(np.uint32)
    for q, t in enumerate(assign):
        o = int(plan.out_offsets[q])
        assert np.array_equal(flat[o:o + shapes[t][1]], orc.answer(ks0[q], Ts[t])), q
    assert all(b.unchanged() for b, _ in guarded) and kbuf.unchanged() and intact(obuf)


def test_materialise_redzones(env):
    torch, pir, orc = env
    rows, B, ld = 3000, 5, 3003
    ks0, _ = make_keys(orc, pir.pir_domain_bits(rows), wl.alphas(80, rows, B), [1] * B, 81)
    kbuf, dkeys = guarded_bytes(torch, b"".join(ks0), 242)
    sbuf = Guarded(torch, B * ld, 343)
    S = sbuf.words().view(B, ld)
    pir.pir_expand_materialise(rows, dkeys, B, S)
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint32)
    init = sbuf.host[GUARD:GUARD + B * ld].reshape(B, ld)
    for q in range(B):
        assert np.array_equal(got[q, :rows], orc.full_eval(ks0[q], rows)), q
    assert np.array_equal(got[:, rows:], init[:, rows:])  # the row padding past `rows` is not written
    assert kbuf.unchanged() and intact(sbuf)


@pytest.mark.parametrize("engine", [0, 1, 2, 3, 4], ids=["imad", "mma_u8", "scan", "tc_f16", "auto"])
@pytest.mark.parametrize("B,L,W,lpad,tpad", [(20, 5000, 64, 4, 4), (130, 3001, 40, 4, 8), (7, 777, 12, 4, 4),
                                             (37, 2048, 33, 3, 1)])
def test_contract_redzones(env, B, L, W, lpad, tpad, engine):
    torch, pir, orc = env
    aligned = W % 4 == 0 and lpad % 4 == 0 and tpad % 4 == 0 and L % 4 == 0
    if engine == 2 and not aligned:
        pytest.skip("the scan engine needs 16-byte rows")
    rng = np.random.Generator(np.random.PCG64(B + L + W))
    Sh = rng.integers(0, 1 << 32, (B, L), dtype=np.uint64).astype(np.uint32)
    T = wl.table_u32(W + 9, L, W)
    ld = L + lpad
    full = rng.integers(0, 1 << 32, (B, ld), dtype=np.uint64).astype(np.uint32)
    full[:, :L] = Sh
    sbuf = Guarded(torch, B * ld, 353, full)
    tbuf, table = guarded_table(torch, T, tpad, 151)
    obuf, out = guarded_out(torch, B, W, 363)
    pir.pir_contract_u32(sbuf.words().view(B, ld)[:, :L], B, table, out, engine=engine)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.contract(Sh, T))
    assert sbuf.unchanged() and tbuf.unchanged() and intact(obuf)
    assert pir.pir_device_status(clear=True) == 0


def test_noalloc_entry_point_redzones(env):
    """The allocation-free entry point reads a guarded, row-padded table."""
    torch, pir, orc = env
    rows, W, B = 3000, 16, 4
    T = wl.table_u32(91, rows, W)
    ks0, _ = make_keys(orc, pir.pir_domain_bits(rows), wl.alphas(92, rows, B), [1] * B, 93)
    tbuf, table = guarded_table(torch, T, 4, 161)
    out = np.zeros((B, W), np.uint32)
    pir.pir_server_eval_noalloc(table, b"".join(ks0), B, out)
    assert np.array_equal(out, _answers(orc, ks0, T))
    assert tbuf.unchanged()


def test_serving_redzones(env):
    """Tables registered with a server are read, never written, and only
    within their rows and widths, whatever the batch mix."""
    torch, pir, orc = env
    shapes, pads = [(2000, 16), (1 << 12, 32), (700, 8)], [4, 8, 4]
    Ts = [wl.table_u32(170 + i, r, w) for i, (r, w) in enumerate(shapes)]
    guarded = [guarded_table(torch, T, p, 171 + i) for i, (T, p) in enumerate(zip(Ts, pads))]
    srv = pir.pir_server_create(max_batch=64)
    try:
        tids = [srv.register_table(v) for _, v in guarded]
        rng = np.random.Generator(np.random.PCG64(172))
        reqs = []
        for q in range(30):
            t = int(rng.integers(0, len(shapes)))
            rows, W = shapes[t]
            k0, _ = make_keys(orc, pir.pir_domain_bits(rows), [int(rng.integers(0, rows))], [1], 180 + q)
            out = np.zeros(W, np.uint32)
            reqs.append((t, k0[0], out, srv.submit(tids[t], k0[0], out)))
        srv.drain()
        for t, key, out, ticket in reqs:
            assert srv.poll(ticket) is not None
            assert np.array_equal(out, orc.answer(key, Ts[t]))
    finally:
        srv.close()
    assert all(b.unchanged() for b, _ in guarded)
