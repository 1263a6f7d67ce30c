"""Parity of the CUDA fused path with the oracle: bit-exact u32 shares.

Keys come from the oracle's Gen with seeded randomness (workloads); tables
from the seeded SplitMix64 generator.  Every share is compared element by
element with the oracle's T x Eval(k, .) mod 2^32, and shares of the two
servers must reconstruct beta * T[alpha] (Sec. 3.1).
"""
import numpy as np
import pytest

import workloads as wl

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


def make_keys(orc, n, alphas, betas, seed):
    rnd = wl.key_randomness(seed, n, len(alphas))
    ks0, ks1 = [], []
    for (r0, r1, c0), a, b in zip(rnd, alphas, betas):
        k0, k1 = orc.gen(n, int(a), int(b), r0, r1, c0)
        ks0.append(k0)
        ks1.append(k1)
    return ks0, ks1


def dev_table(torch, T):
    return torch.from_numpy(np.ascontiguousarray(T).view(np.int32)).cuda()


def dev_keys(torch, keys):
    return torch.frombuffer(bytearray(b"".join(keys)), dtype=torch.uint8).cuda()


def run_device(torch, pir, table, keys, W, plan=None, status=None):
    dk = dev_keys(torch, keys)
    out = torch.empty((len(keys), W), dtype=torch.int32, device="cuda")
    if plan is None:
        pir.pir_server_eval_device(table, dk, len(keys), out, status)
    else:
        pir.pir_server_eval_device_plan(table, dk, len(keys), out, plan, status)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


SHAPES = [  # (rows, width, batch): several tiles and ragged tails
    (2, 1, 1), (3, 4, 2), (100, 3, 5), (1000, 16, 9), (4096 + 77, 16, 3), (1 << 14, 64, 8),
    ((1 << 15) + 1000, 32, 11), (1 << 12, 1, 17), (1 << 13, 100, 4), (1 << 11, 256, 8),
    (5000, 4, 5), (3000, 8, 9),  # narrow aligned rows: one or two column chunks per consumer row group
]


@pytest.mark.parametrize("rows,width,batch", SHAPES)
def test_fused_matches_oracle(env, rows, width, batch):
    torch, pir, orc = env
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(rows * 7 + width, rows, width)
    alphas = wl.alphas(rows, rows, batch)
    alphas[0] = rows - 1
    betas = [1] * batch
    if batch > 1:
        betas[1] = M32
    ks0, ks1 = make_keys(orc, n, alphas, betas, rows + batch)
    table = dev_table(torch, T)
    g0 = run_device(torch, pir, table, ks0, width)
    g1 = run_device(torch, pir, table, ks1, width)
    for q in range(batch):
        assert np.array_equal(g0[q], orc.answer(ks0[q], T)), q
        assert np.array_equal(g1[q], orc.answer(ks1[q], T)), q
        want = (T[alphas[q]].astype(np.uint64) * betas[q]) & M32
        assert np.array_equal(pir.pir_reconstruct(g0[q], g1[q]), want.astype(np.uint32))


def test_every_launch_shape_matches_oracle(env):
    # every (group, load width, rows per item) the library accepts for this shape
    torch, pir, orc = env
    rows, width, batch = (1 << 13) + 333, 16, 9
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(21, rows, width)
    alphas = wl.alphas(3, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 77)
    want = np.stack([orc.answer(k, T) for k in ks0])
    table = dev_table(torch, T)
    ran = 0
    for g in (1, 2, 4, 8):
        for vec in (1, 4):
            for r in range(1, n + 1):
                plan = pir.pir_plan(g, r, vec, 0)
                try:
                    got = run_device(torch, pir, table, ks0, width, plan=plan)
                except pir.PirError as e:
                    assert e.code == -8, plan.as_dict()  # shape outside the kernels' limits
                    continue
                assert np.array_equal(got, want), plan.as_dict()
                ran += 1
    assert ran >= 80


def test_cut_last_round_matches_oracle(env):
    # Items that do not fill the grid's last round are cut into 2^tail_log2
    # pieces: every forced cut gives the oracle's shares, the ragged last
    # range (pieces past the last row are skipped) included.
    torch, pir, orc = env
    rows, width, batch = (1 << 13) + 333, 16, 9
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(23, rows, width)
    alphas = wl.alphas(5, rows, batch)
    alphas[0] = rows - 1
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 78)
    want = np.stack([orc.answer(k, T) for k in ks0])
    table = dev_table(torch, T)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cut = 0
    for g in (1, 2, 8):
        for r in range(2, 9):
            for s in range(1, min(3, r - 1) + 1):
                plan = pir.pir_plan(g, r, 4, 0)
                plan.tail_log2 = s
                got = run_device(torch, pir, table, ks0, width, plan=plan)
                assert np.array_equal(got, want), plan.as_dict()
                items = -(-rows // (1 << r)) * -(-batch // g)
                cut += items > sms and items % sms != 0
    assert cut >= 10
    plan = pir.pir_plan(1, 3, 4, 0)
    plan.tail_log2 = 3  # pieces of 2^0 rows: outside the kernels' limits
    with pytest.raises(pir.PirError) as e:
        run_device(torch, pir, table, ks0, width, plan=plan)
    assert e.value.code == -8


def test_planner_cut_for_fused_and_expand(env):
    # 200 queries over 2^14 + 77 rows: on 152 SMs the cost model takes items of
    # 2^11 rows and 8 queries (225 items) and cuts the 73 of the last round in
    # halves.  Both the fused product and the expansion equal the oracle.
    torch, pir, orc = env
    rows, width, batch = (1 << 14) + 77, 16, 200
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(29, rows, width)
    alphas = wl.alphas(29, rows, batch)
    alphas[-1] = rows - 1
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 29)
    plan = pir.pir_plan_for(rows, width, batch)
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        assert (plan.group, plan.range_log2, plan.tail_log2) == (8, 11, 1), plan.as_dict()
    Y = np.stack([orc.full_eval(k, rows) for k in ks0])
    table = dev_table(torch, T)
    got = run_device(torch, pir, table, ks0, width)
    assert np.array_equal(got, orc.contract(Y, T))
    dk = dev_keys(torch, ks0)
    S = torch.empty((batch, rows + 3), dtype=torch.int32, device="cuda")
    pir.pir_expand_materialise(rows, dk, batch, S)
    torch.cuda.synchronize()
    assert np.array_equal(S.cpu().numpy().view(np.uint32)[:, :rows], Y)


def test_autotuned_plan_is_used_and_exact(env):
    torch, pir, orc = env
    rows, width, batch = (1 << 15) + 9, 32, 12
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(44, rows, width)
    alphas = wl.alphas(44, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 44)
    table = dev_table(torch, T)
    dk = dev_keys(torch, ks0)
    out = torch.empty((batch, width), dtype=torch.int32, device="cuda")
    plan, ms = pir.pir_autotune(table, dk, batch, out)
    assert ms > 0 and plan.group in (1, 2, 4, 8) and 1 <= plan.range_log2 <= n
    chosen = pir.pir_plan_for(rows, width, batch)  # the cache answers for this shape now
    assert (chosen.group, chosen.range_log2, chosen.vec) == (plan.group, plan.range_log2, plan.vec)
    got = run_device(torch, pir, table, ks0, width)
    for q in range(batch):
        assert np.array_equal(got[q], orc.answer(ks0[q], T))


def test_autotuner_weighs_expand_and_scan_for_few_queries(env):
    """For a few queries the autotuner also times the expand-and-scan strategy;
    whichever it keeps, pir_plan_for reports it and the evaluation equals the
    oracle.  An explicit plan of either strategy gives the same shares."""
    torch, pir, orc = env
    rows, width, batch = 1 << 18, 64, 2
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(45, rows, width)
    alphas = wl.alphas(45, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 45)
    table = dev_table(torch, T)
    dk = dev_keys(torch, ks0)
    out = torch.empty((batch, width), dtype=torch.int32, device="cuda")
    plan, ms = pir.pir_autotune(table, dk, batch, out)
    assert ms > 0 and plan.strategy in (pir.PIR_STRATEGY_FUSED, pir.PIR_STRATEGY_EXPAND_SCAN,
                                        pir.PIR_STRATEGY_FUSED_STAGED)
    chosen = pir.pir_plan_for(rows, width, batch)
    assert (chosen.strategy, chosen.group, chosen.range_log2) == (plan.strategy, plan.group, plan.range_log2)
    got = run_device(torch, pir, table, ks0, width)
    for q in range(batch):
        assert np.array_equal(got[q], orc.answer(ks0[q], T))
    fused = pir.pir_plan_for(rows, width, batch)
    fused.strategy = pir.PIR_STRATEGY_FUSED
    scan = pir.pir_plan_for(rows, width, batch)
    scan.strategy = pir.PIR_STRATEGY_EXPAND_SCAN
    if fused.group > batch:
        fused.group = 2
    assert np.array_equal(run_device(torch, pir, table, ks0, width, plan=fused), got)
    assert np.array_equal(run_device(torch, pir, table, ks0, width, plan=scan), got)


def test_host_entry_point_host_and_device_outputs(env):
    torch, pir, orc = env
    rows, width, batch = 5000, 8, 6
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(8, rows, width)
    alphas = wl.alphas(8, rows, batch)
    ks0, ks1 = make_keys(orc, n, alphas, [1] * batch, 8)
    table = dev_table(torch, T)
    host_out = np.zeros((batch, width), np.uint32)
    pir.pir_server_eval(table, b"".join(ks0), batch, host_out)
    dev_out = torch.zeros((batch, width), dtype=torch.int32, device="cuda")
    pir.pir_server_eval(table, b"".join(ks1), batch, dev_out)
    torch.cuda.synchronize()
    d1 = dev_out.cpu().numpy().view(np.uint32)
    for q in range(batch):
        assert np.array_equal(host_out[q], orc.answer(ks0[q], T))
        assert np.array_equal(d1[q], orc.answer(ks1[q], T))


def test_host_entry_rejects_bad_keys_and_domains(env):
    torch, pir, orc = env
    T = wl.table_u32(1, 300, 4)
    table = dev_table(torch, T)
    k0, _ = make_keys(orc, 9, [5], [1], 1)
    out = np.zeros((1, 4), np.uint32)
    bad = bytearray(k0[0])
    bad[0] ^= 1
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval(table, bytes(bad), 1, out)
    assert e.value.code == -3
    k_wrong, _ = make_keys(orc, 10, [5], [1], 1)
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval(table, k_wrong[0], 1, out)
    assert e.value.code in (-2, -3)


def test_device_status_flags_bad_key_and_zeroes_its_share(env):
    torch, pir, orc = env
    rows, width = 3000, 16
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(2, rows, width)
    ks0, _ = make_keys(orc, n, [1, 2, 3, 4], [1] * 4, 2)
    bad = bytearray(ks0[2])
    bad[6] = 7  # party out of range
    keys = [ks0[0], ks0[1], bytes(bad), ks0[3]]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = run_device(torch, pir, dev_table(torch, T), keys, width, status=status)
    assert int(status.item()) & pir.PIR_STATUS_BAD_KEY
    assert not got[2].any()
    for q in (0, 1, 3):
        assert np.array_equal(got[q], orc.answer(ks0[q], T))


def test_range_shards_sum_to_full_and_match_oracle(env):
    # Sec. 3.2.7: shards over index ranges, summed, equal the full share.
    torch, pir, orc = env
    rows, width, batch = (1 << 14) + 100, 16, 5
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(4, rows, width)
    alphas = wl.alphas(4, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 4)
    dk = dev_keys(torch, ks0)
    table = dev_table(torch, T)
    cuts = [0, 1, 4096, 4097, 10000, rows]
    total = np.zeros((batch, width), np.uint64)
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        out = torch.empty((batch, width), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_range(table[lo:hi], lo, rows, dk, batch, out)
        torch.cuda.synchronize()
        part = out.cpu().numpy().view(np.uint32)
        for q in range(batch):
            assert np.array_equal(part[q], orc.answer(ks0[q], T, lo, hi)), (lo, hi, q)
        total += part
    total = (total & M32).astype(np.uint32)
    for q in range(batch):
        assert np.array_equal(total[q], orc.answer(ks0[q], T))


def test_degenerate_domains_and_extreme_betas(env):
    torch, pir, orc = env
    for rows, width in ((2, 1), (2, 4), (3, 1), (5, 2)):
        n = pir.pir_domain_bits(rows)
        T = wl.table_u32(rows, rows, width)
        table = dev_table(torch, T)
        for alpha in (0, rows - 1):
            for beta in (0, 1, M32):
                ks0, ks1 = make_keys(orc, n, [alpha], [beta], alpha * 3 + rows)
                g0 = run_device(torch, pir, table, ks0, width)
                g1 = run_device(torch, pir, table, ks1, width)
                assert np.array_equal(g0[0], orc.answer(ks0[0], T))
                assert np.array_equal(g1[0], orc.answer(ks1[0], T))
                want = (T[alpha].astype(np.uint64) * beta) & M32
                assert np.array_equal(pir.pir_reconstruct(g0[0], g1[0]), want.astype(np.uint32))


def test_library_keys_on_gpu_reconstruct(env):
    torch, pir, _ = env
    rows, width, batch = 1 << 12, 16, 8
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(6, rows, width)
    alphas = wl.alphas(6, rows, batch)
    pairs = [pir.pir_keygen(n, int(a), 1, None) for a in alphas]
    table = dev_table(torch, T)
    g0 = run_device(torch, pir, table, [p[0] for p in pairs], width)
    g1 = run_device(torch, pir, table, [p[1] for p in pairs], width)
    for q in range(batch):
        assert np.array_equal(pir.pir_reconstruct(g0[q], g1[q]), T[alphas[q]])


def test_host_entry_point_repeated_calls_and_streams(env):
    """Small synchronous calls run through one staging area per host thread
    and device, as a graph kept per call shape (table, batch, plan), whose
    one copy in brings the keys and a zeroed share area: calls of growing and
    shrinking widths and batches on new tables (more shapes than the graphs
    kept, so some are dropped and rebuilt), on two streams in turn, then one
    shape again and again with new keys and the table's contents replaced in
    place; each share matches the oracle word for word (stale keys, a share
    area not cleared, or a graph holding old contents would show up here)."""
    torch, pir, orc = env
    streams = [torch.cuda.Stream(), torch.cuda.current_stream()]
    cases = [(3000, 8, 1), (3000, 64, 3), (5000, 16, 7), (3000, 8, 2), (1 << 12, 128, 4), (5000, 16, 1)]
    for i, (rows, width, batch) in enumerate(cases * 2):
        n = pir.pir_domain_bits(rows)
        T = wl.table_u32(rows + width, rows, width)
        ks0, _ = make_keys(orc, n, wl.alphas(i, rows, batch), [1] * batch, 90 + i)
        out = np.full((batch, width), 0x5A5A5A5A, np.uint32)
        pir.pir_server_eval(dev_table(torch, T), b"".join(ks0), batch, out, stream=streams[i % 2])
        for q in range(batch):
            assert np.array_equal(out[q], orc.answer(ks0[q], T)), (i, q)
    rows, width = 5000, 16
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(77, rows, width)
    table = dev_table(torch, T)
    for i in range(8):
        if i == 4:
            T = wl.table_u32(78, rows, width)
            table.copy_(dev_table(torch, T))
        batch = 1 + (i % 2)
        ks0, _ = make_keys(orc, n, wl.alphas(200 + i, rows, batch), [1] * batch, 300 + i)
        out = np.full((batch, width), 0x5A5A5A5A, np.uint32)
        pir.pir_server_eval(table, b"".join(ks0), batch, out, stream=streams[i % 2])
        for q in range(batch):
            assert np.array_equal(out[q], orc.answer(ks0[q], T)), (i, q)


def test_host_entry_point_at_the_staging_limits(env):
    """The host call stages keys and shares of up to 32 KiB each in the calling
    thread's buffers (one graph per shape) and takes the stream-ordered pool
    beyond that: calls just inside both limits and just past each of them
    give the oracle's shares word for word, on both sides twice."""
    torch, pir, orc = env
    rows = 1 << 16
    n = pir.pir_domain_bits(rows)
    kb = pir.pir_key_bytes(n)
    inside = (32 << 10) // kb  # keys just inside 32 KiB
    cases = [(inside, 8), (inside + 1, 8),  # key bytes: staged, then pooled
             (8, 1024), (9, 1024)]  # share bytes: 32 KiB, then past it (1024 words: the widest fused rows)
    for i, (batch, width) in enumerate(cases * 2):
        T = wl.table_u32(700 + width, rows, width)
        table = dev_table(torch, T)
        ks0, _ = make_keys(orc, n, wl.alphas(710 + i, rows, batch), [1] * batch, 720 + i)
        out = np.full((batch, width), 0x5A5A5A5A, np.uint32)
        pir.pir_server_eval(table, b"".join(ks0), batch, out)
        for q in sorted({0, batch // 2, batch - 1}):
            assert np.array_equal(out[q], orc.answer(ks0[q], T)), (i, batch, width, q)


def test_single_group_launches_overwrite_every_share(env):
    """Launches whose batch is one query group (a lone query, or up to 8
    queries) accumulate every CTA's sums into the output: outputs filled with
    garbage first come back as the oracle's shares (the output is cleared in
    stream order before the kernel adds into it), on repeated launches over
    two streams, for an index-range shard too, and a bad key's share is zero."""
    torch, pir, orc = env
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rows, width, batch in [(1 << 16, 16, 1), (5000, 8, 2), (1 << 14, 64, 8), ((1 << 13) + 5, 4, 4)]:
        n = pir.pir_domain_bits(rows)
        T = wl.table_u32(rows + 2 * width, rows, width)
        ks0, _ = make_keys(orc, n, wl.alphas(rows + 9, rows, batch), [1] * batch, rows + 11)
        keys = list(ks0)
        if batch > 1:
            bad = bytearray(keys[-1])
            bad[0] ^= 0xFF  # magic
            keys[-1] = bytes(bad)
        table = dev_table(torch, T)
        dk = dev_keys(torch, keys)
        want = [orc.answer(k, T) for k in keys[:batch - 1 if batch > 1 else 1]]
        for rep in range(4):
            st = streams[rep % 2]
            out = torch.full((batch, width), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
            with torch.cuda.stream(st):
                pir.pir_server_eval_device(table, dk, batch, out, stream=st)
            st.synchronize()
            got = out.cpu().numpy().view(np.uint32)
            for q, w in enumerate(want):
                assert np.array_equal(got[q], w), (rows, batch, rep, q)
            if batch > 1:
                assert not got[-1].any()
    # an index-range shard with one query: rows [lo, hi) of a 5000-row domain
    L, W, lo, hi = 5000, 16, 1024, 3000
    T = wl.table_u32(77, L, W)
    ks0, _ = make_keys(orc, pir.pir_domain_bits(L), [2500], [1], 78)
    out = torch.full((1, W), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    pir.pir_server_eval_range(dev_table(torch, T[lo:hi]), lo, L, dev_keys(torch, ks0), 1, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], orc.answer(ks0[0], T, lo, hi))
