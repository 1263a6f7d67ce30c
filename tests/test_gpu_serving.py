"""The serving loop: every result is the same whether its query ran alone or
in a mixed batch with other tables' queries, and equals the oracle's share;
admission refuses when the pool is full; Poisson replay reconstructs every
row."""
import time

import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_table, make_keys

pytestmark = pytest.mark.gpu
M32 = 0xFFFFFFFF
SHAPES = [(3000, 16), (1 << 12, 64), (1 << 14, 32), (777, 8)]


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import oracle
    import paper_2301_10904_gb300 as pir

    Ts = [wl.table_u32(500 + i, r, w) for i, (r, w) in enumerate(SHAPES)]
    dts = [dev_table(torch, T) for T in Ts]
    return torch, pir, oracle, Ts, dts


def _wait(srv, ticket, timeout=30.0):
    t0 = time.time()
    while True:
        lat = srv.poll(ticket)
        if lat is not None:
            return lat
        assert time.time() - t0 < timeout, "query did not finish"
        time.sleep(0.0005)


def test_each_result_same_alone_and_in_the_mix(env):
    torch, pir, orc, Ts, dts = env
    srv = pir.Server(max_batch=64, streams=2)
    tids = [srv.register_table(t) for t in dts]
    rng = np.random.Generator(np.random.PCG64(8))
    assign = rng.integers(0, len(SHAPES), 40).tolist()
    queries = []
    for q, t in enumerate(assign):
        n = pir.pir_domain_bits(SHAPES[t][0])
        alpha = int(rng.integers(0, SHAPES[t][0]))
        k0, _ = make_keys(orc, n, [alpha], [1], 900 + q)
        queries.append((t, k0[0]))
    alone = []
    for t, k in queries:  # one at a time: each is a batch of its own
        out = np.zeros(SHAPES[t][1], np.uint32)
        _wait(srv, srv.submit(tids[t], k, out))
        alone.append(out)
    mixed = [np.zeros(SHAPES[t][1], np.uint32) for t, _ in queries]
    tickets = [srv.submit(tids[t], k, o) for (t, k), o in zip(queries, mixed)]  # all at once
    for tk in tickets:
        _wait(srv, tk)
    st = srv.stats()
    assert st["batches"] < 2 * len(queries)  # the mixed submission was batched
    for (t, k), a, m in zip(queries, alone, mixed):
        assert np.array_equal(a, m)
        assert np.array_equal(m, orc.answer(k, Ts[t]))
    srv.close()


def test_admission_refuses_when_pool_is_full(env):
    torch, pir, orc, Ts, dts = env
    srv = pir.Server(max_inflight=2)
    tid = srv.register_table(dts[0])
    n = pir.pir_domain_bits(SHAPES[0][0])
    ks, _ = make_keys(orc, n, [1, 2, 3], [1, 1, 1], 5)
    outs = [np.zeros(SHAPES[0][1], np.uint32) for _ in range(3)]
    t0 = srv.submit(tid, ks[0], outs[0])
    t1 = srv.submit(tid, ks[1], outs[1])
    with pytest.raises(pir.PirError) as e:  # both slots held until polled
        srv.submit(tid, ks[2], outs[2])
    assert e.value.code == -7
    _wait(srv, t0)
    t2 = srv.submit(tid, ks[2], outs[2])  # a released slot admits the next query
    _wait(srv, t1)
    _wait(srv, t2)
    for k, o in zip(ks, outs):
        assert np.array_equal(o, orc.answer(k, Ts[0]))
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_submit_rejects_keys_of_another_domain(env):
    torch, pir, orc, Ts, dts = env
    srv = pir.Server()
    tid = srv.register_table(dts[1])  # 2^12 rows: n = 12
    k, _ = make_keys(orc, 10, [3], [1], 1)
    with pytest.raises(pir.PirError) as e:
        srv.submit(tid, k[0], np.zeros(64, np.uint32))
    assert e.value.code == -2
    srv.close()


def test_poisson_replay_reconstructs_every_row(env):
    torch, pir, orc, Ts, dts = env
    srv = pir.Server(max_batch=256, streams=2)
    tids = [srv.register_table(t) for t in dts]
    count = 400
    arrivals = wl.poisson_arrivals(3, 4000.0, count)
    assign = wl.uniform_tables(3, len(SHAPES), count)
    rng = np.random.Generator(np.random.PCG64(3))
    alphas = [int(rng.integers(0, SHAPES[t][0])) for t in assign]
    keys = ([], [])
    for q, (t, a) in enumerate(zip(assign, alphas)):
        k0, k1 = pir.pir_keygen(pir.pir_domain_bits(SHAPES[t][0]), a, 1, bytes([q & 255, q >> 8, 7]) * 10 + b"xy")
        keys[0].append(k0)
        keys[1].append(k1)
    widths = [SHAPES[t][1] for t in assign]
    out_off = np.concatenate([[0], np.cumsum(widths)[:-1]]).astype(np.uint64)
    shares = []
    for party in (0, 1):
        kbytes = b"".join(keys[party])
        key_off = np.concatenate([[0], np.cumsum([len(k) for k in keys[party]])[:-1]]).astype(np.uint64)
        outs = np.zeros(int(sum(widths)), np.uint32)
        lat, elapsed = srv.replay(arrivals, [tids[t] for t in assign], kbytes, key_off, outs, out_off)
        assert (lat > 0).all() and elapsed > 0
        shares.append(outs)
    for q, t in enumerate(assign):
        o, w = int(out_off[q]), widths[q]
        rec = ((shares[0][o:o + w].astype(np.uint64) + shares[1][o:o + w]) & M32).astype(np.uint32)
        assert np.array_equal(rec, Ts[t][alphas[q]]), q
    srv.close()


def test_serving_mix_at_full_size():
    """The serving workload's four resident tables (2^18 x 64, 2^20 x 32,
    2^22 x 32, 2^24 x 16 words; 1.73 GB) in the server's own launch
    configuration: 256 Poisson queries, table uniform per query, both servers;
    every query reconstructs its row, eight queries give the same share alone
    as in the mix, and 16 sampled queries per table match the oracle."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from concurrent.futures import ThreadPoolExecutor
    import os

    import __graft_entry__ as g

    g.build()
    import oracle as orc
    import paper_2301_10904_gb300 as pir

    shapes = wl.SERVING_TABLES
    tables = [wl.table_u32_torch(700 + i, r, w, "cuda") for i, (r, w) in enumerate(shapes)]
    ns = [pir.pir_domain_bits(r) for r, _ in shapes]
    count = 256
    assign = wl.uniform_tables(701, len(shapes), count).tolist()
    rng = np.random.Generator(np.random.PCG64(701))
    alphas = [int(rng.integers(0, shapes[t][0])) for t in assign]
    pairs = [pir.pir_keygen(ns[t], a, 1, bytes([q % 256, q // 256]) * 16) for q, (t, a) in enumerate(zip(assign, alphas))]
    widths = np.array([shapes[t][1] for t in assign], np.uint64)
    ooff = np.concatenate([[0], np.cumsum(widths)[:-1]]).astype(np.uint64)
    klens = np.array([len(p[0]) for p in pairs], np.uint64)
    koff = np.concatenate([[0], np.cumsum(klens)[:-1]]).astype(np.uint64)
    srv = pir.Server(max_batch=2048, streams=2)
    tids = [srv.register_table(t) for t in tables]
    outs = []
    for party in (0, 1):
        keys = b"".join(p[party] for p in pairs)
        o = np.zeros(int(widths.sum()), np.uint32)
        srv.replay(wl.poisson_arrivals(702, 3000, count), [tids[t] for t in assign], keys, koff, o, ooff)
        outs.append(o)
    rec = ((outs[0].astype(np.uint64) + outs[1]) & M32).astype(np.uint32)
    for q in range(count):
        o, w = int(ooff[q]), int(widths[q])
        want = tables[assign[q]][alphas[q]].cpu().numpy().view(np.uint32)
        assert np.array_equal(rec[o:o + w], want), q
    # the same share alone as in the mix
    picks = [next(q for q in range(count) if assign[q] == t) for t in range(len(shapes))]
    picks += [next(q for q in range(count - 1, -1, -1) if assign[q] == t) for t in range(len(shapes))]
    for q in picks:
        alone = np.zeros(int(widths[q]), np.uint32)
        _wait(srv, srv.submit(tids[assign[q]], pairs[q][0], alone), timeout=60.0)
        assert np.array_equal(alone, outs[0][int(ooff[q]):int(ooff[q]) + int(widths[q])]), q
    srv.close()
    # 16 queries per table against the oracle, in parallel host threads (one
    # 2^24-row expansion takes the oracle tens of seconds)
    host = [t.cpu().numpy().view(np.uint32) for t in tables]
    sample = []
    for t in range(len(shapes)):
        qs = [q for q in range(count) if assign[q] == t]
        sample += qs[:: max(1, len(qs) // 16)][:16]
    with ThreadPoolExecutor(max(1, min(len(sample), os.cpu_count() or 1))) as ex:
        got = list(ex.map(lambda q: orc.answer(pairs[q][0], host[assign[q]]), sample))
    for q, want in zip(sample, got):
        assert np.array_equal(outs[0][int(ooff[q]):int(ooff[q]) + int(widths[q])], want), q


def test_batch_buffers_presized_and_grown_in_stream_order(env):
    # Slots are sized for max_batch queries at start: an ordinary mix does not
    # reallocate. Tiny items (2^2 rows: up to 4,096 work items per query on the
    # 2^14-row table) outgrow that estimate; the slots grow (stream-ordered,
    # while the other stream's batch may run) and every share stays the oracle's.
    torch, pir, orc, Ts, dts = env
    for item_log2, expect_growth in ((0, False), (2, True)):
        srv = pir.Server(max_batch=4, streams=2, item_log2=item_log2)
        tids = [srv.register_table(t) for t in dts]
        rng = np.random.Generator(np.random.PCG64(77 + item_log2))
        assign = rng.integers(0, len(SHAPES), 24).tolist()
        outs, wants = [], []
        tickets = []
        for q, t in enumerate(assign):
            n = pir.pir_domain_bits(SHAPES[t][0])
            alpha = int(rng.integers(0, SHAPES[t][0]))
            k0, _ = make_keys(orc, n, [alpha], [1], 4000 + 100 * item_log2 + q)
            out = np.zeros(SHAPES[t][1], np.uint32)
            tickets.append(srv.submit(tids[t], k0[0], out))
            outs.append(out)
            wants.append(orc.answer(k0[0], Ts[t]))
        for tk in tickets:
            _wait(srv, tk, timeout=60.0)
        st = srv.stats()
        srv.close()
        for q in range(len(assign)):
            assert np.array_equal(outs[q], wants[q]), (item_log2, q)
        assert (st["grows"] > 0) == expect_growth, st
