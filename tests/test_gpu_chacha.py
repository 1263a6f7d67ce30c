"""The ChaCha20 PRF on the GPU (the alternative PRF of Sec. 3.2.6, Table 5):
fused, materialised, multi-table and mixed-PRF batches against the oracle, and
mixed-PRF keys through serving, range shards, the allocation-free entry point
and the expand-and-scan strategy."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_keys, dev_table, run_device

pytestmark = pytest.mark.gpu
M32 = 0xFFFFFFFF


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


def _keys(orc, n, alphas, prfs, seed):
    ks0, ks1 = [], []
    for (r0, r1, c0), a, prf in zip(wl.key_randomness(seed, n, len(alphas)), alphas, prfs):
        k0, k1 = orc.gen(n, int(a), 1, r0, r1, c0, prf)
        ks0.append(k0)
        ks1.append(k1)
    return ks0, ks1


@pytest.mark.parametrize("rows,width,batch", [(2, 1, 1), (1000, 16, 9), (1 << 14, 64, 8), ((1 << 15) + 7, 32, 3)])
def test_chacha_fused_matches_oracle(env, rows, width, batch):
    torch, pir, orc = env
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(rows + 11, rows, width)
    alphas = wl.alphas(rows + 11, rows, batch)
    ks0, ks1 = _keys(orc, n, alphas, [1] * batch, rows)
    table = dev_table(torch, T)
    g0 = run_device(torch, pir, table, ks0, width)
    g1 = run_device(torch, pir, table, ks1, width)
    for q in range(batch):
        assert np.array_equal(g0[q], orc.answer(ks0[q], T)), q
        rec = ((g0[q].astype(np.uint64) + g1[q]) & M32).astype(np.uint32)
        assert np.array_equal(rec, T[alphas[q]])


def test_mixed_prf_batch_and_materialised(env):
    torch, pir, orc = env
    rows, width, batch = 5000, 16, 12
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(3, rows, width)
    alphas = wl.alphas(3, rows, batch)
    prfs = [q % 2 for q in range(batch)]  # AES and ChaCha20 queries in one launch
    ks0, _ = _keys(orc, n, alphas, prfs, 30)
    table = dev_table(torch, T)
    got = run_device(torch, pir, table, ks0, width)
    S = torch.empty((batch, rows), dtype=torch.int32, device="cuda")
    pir.pir_expand_materialise(rows, dev_keys(torch, ks0), batch, S)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy().view(np.uint32)
    for q in range(batch):
        assert np.array_equal(got[q], orc.answer(ks0[q], T)), q
        assert np.array_equal(Sh[q], orc.full_eval(ks0[q], rows)), q


def test_chacha_multi_table_and_library_keys(env):
    torch, pir, orc = env
    shapes = [(3000, 16), (1 << 13, 32)]
    Ts = [wl.table_u32(70 + i, r, w) for i, (r, w) in enumerate(shapes)]
    dts = [dev_table(torch, T) for T in Ts]
    assign = [0, 1, 1, 0, 1, 0, 0, 1, 1, 1]
    rng = np.random.Generator(np.random.PCG64(70))
    alphas = [int(rng.integers(0, shapes[t][0])) for t in assign]
    pairs = [pir.pir_keygen_prf(pir.pir_domain_bits(shapes[t][0]), a, 1, pir.PIR_PRF_CHACHA20 if q % 3 else 0,
                                bytes([q]) * 32) for q, (t, a) in enumerate(zip(assign, alphas))]
    plan = pir.pir_multi_plan_create(dts, assign)
    outs = []
    for party in (0, 1):
        buf = bytearray(plan.key_bytes_total)
        for q, p in enumerate(pairs):
            o = int(plan.key_offsets[q])
            buf[o:o + len(p[party])] = p[party]
        out = torch.empty((plan.out_words_total,), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_multi(plan, torch.frombuffer(buf, dtype=torch.uint8).cuda(), out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().view(np.uint32))
    for q, t in enumerate(assign):
        o, w = int(plan.out_offsets[q]), shapes[t][1]
        rec = ((outs[0][o:o + w].astype(np.uint64) + outs[1][o:o + w]) & M32).astype(np.uint32)
        assert np.array_equal(rec, Ts[t][alphas[q]]), q
        assert np.array_equal(outs[0][o:o + w], orc.answer(pairs[q][0], Ts[t])), q


def test_mixed_prf_every_path_and_split_shape(env):
    # Explicit plans from whole-table items (no path walk) down to 2-row items
    # (a 12-level path walk), every query-slot count: the dependent levels compute
    # one child per thread for both PRFs, and a malformed key still yields a zero
    # share and the status flag.
    torch, pir, orc = env
    rows, width, batch = (1 << 12) + 5, 16, 9
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(91, rows, width)
    alphas = wl.alphas(91, rows, batch)
    alphas[2] = rows - 1
    ks0, _ = _keys(orc, n, alphas, [q % 2 for q in range(batch)], 91)
    bad = bytearray(ks0[4])
    bad[6] = 9  # party out of range
    keys = ks0[:4] + [bytes(bad)] + ks0[5:]
    want = [orc.answer(k, T) for k in ks0]
    table = dev_table(torch, T)
    ran = 0
    for g in (1, 2, 4, 8):
        for r in (1, 2, 4, 7, 10, n):
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            got = run_device(torch, pir, table, keys, width, plan=pir.pir_plan(g, r, 4, 0), status=status)
            assert int(status.item()) & pir.PIR_STATUS_BAD_KEY, (g, r)
            assert not got[4].any(), (g, r)
            for q in range(batch):
                if q != 4:
                    assert np.array_equal(got[q], want[q]), (g, r, q)
            ran += 1
    assert ran == 24


def test_mixed_prf_serving_shards_noalloc_and_expand_scan(env):
    """Keys of both PRFs through the entry points not covered above: the
    serving loop, index-range shards summed over the table, the
    allocation-free entry point and the expand-and-scan strategy; every
    share equals the oracle's and both parties reconstruct T[alpha]."""
    torch, pir, orc = env
    rows, width, batch = 5000, 16, 6
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(95, rows, width)
    alphas = wl.alphas(95, rows, batch)
    ks0, ks1 = _keys(orc, n, alphas, [q % 2 for q in range(batch)], 95)
    table = dev_table(torch, T)
    for keys in (ks0, ks1):
        want = np.stack([orc.answer(k, T) for k in keys])
        # expand-and-scan strategy on an explicit plan
        plan = pir.pir_plan_for(rows, width, batch)
        plan.strategy = pir.PIR_STRATEGY_EXPAND_SCAN
        got = run_device(torch, pir, table, keys, width, plan=plan)
        assert np.array_equal(got, want)
        # index-range shards, summed mod 2^32
        dk = dev_keys(torch, keys)
        total = np.zeros((batch, width), np.uint64)
        for lo, hi in ((0, 1024), (1024, 3000), (3000, rows)):
            part = torch.empty((batch, width), dtype=torch.int32, device="cuda")
            pir.pir_server_eval_range(table[lo:hi], lo, rows, dk, batch, part)
            torch.cuda.synchronize()
            total += part.cpu().numpy().view(np.uint32)
        assert np.array_equal((total & M32).astype(np.uint32), want)
        # allocation-free entry point
        out = np.zeros((batch, width), np.uint32)
        pir.pir_server_eval_noalloc(table, b"".join(keys), batch, out)
        assert np.array_equal(out, want)
        # serving loop
        srv = pir.pir_server_create(max_batch=16)
        try:
            tid = srv.register_table(table)
            outs = [np.zeros(width, np.uint32) for _ in keys]
            tickets = [srv.submit(tid, k, o) for k, o in zip(keys, outs)]
            srv.drain()
            assert all(srv.poll(t) is not None for t in tickets)
            assert np.array_equal(np.stack(outs), want)
        finally:
            srv.close()
    rec0 = np.stack([orc.answer(k, T) for k in ks0]).astype(np.uint64)
    rec1 = np.stack([orc.answer(k, T) for k in ks1]).astype(np.uint64)
    assert np.array_equal(((rec0 + rec1) & M32).astype(np.uint32), T[alphas])
