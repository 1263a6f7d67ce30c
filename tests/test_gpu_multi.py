"""Many tables of uneven sizes and widths in one persistent launch: every
query's share against the oracle, CUDA-graph replay, the autotuner, bad keys,
and the full-size 8-table Zipf mix."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_table, make_keys

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


def _mix(torch, pir, orc, shapes, assign, seed):
    """Host tables, device tables, per-query keys (both parties) and the packed
    device key buffers for a plan's layout."""
    Ts = [wl.table_u32(seed + i, r, w) for i, (r, w) in enumerate(shapes)]
    dts = [dev_table(torch, T) for T in Ts]
    ns = [pir.pir_domain_bits(r) for r, _ in shapes]
    rng = np.random.Generator(np.random.PCG64(seed))
    alphas = np.array([rng.integers(0, shapes[t][0]) for t in assign], np.uint64)
    ks0, ks1 = [], []
    for q, t in enumerate(assign):
        k0, k1 = make_keys(orc, ns[t], [alphas[q]], [1], seed * 1000 + q)
        ks0.append(k0[0])
        ks1.append(k1[0])
    return Ts, dts, alphas, ks0, ks1


def _pack(torch, plan, keys):
    buf = bytearray(plan.key_bytes_total)
    for q, k in enumerate(keys):
        o = int(plan.key_offsets[q])
        buf[o:o + len(k)] = k
    return torch.frombuffer(buf, dtype=torch.uint8).cuda()


def _unpack(plan, out, shapes, assign):
    flat = out.cpu().numpy().view(np.uint32)
    return [flat[int(plan.out_offsets[q]):int(plan.out_offsets[q]) + shapes[t][1]] for q, t in enumerate(assign)]


SHAPES = [(1000, 16), (4096, 4), (1 << 13, 64), (3, 8), (2500, 32), (1 << 14, 128)]


@pytest.mark.parametrize("item_log2", [0, 9, 12])
def test_multi_matches_oracle(env, item_log2):
    torch, pir, orc = env
    rng = np.random.Generator(np.random.PCG64(5))
    assign = rng.choice([0, 1, 2, 3, 5], size=29).tolist()  # table 4 gets no queries
    Ts, dts, alphas, ks0, ks1 = _mix(torch, pir, orc, SHAPES, assign, 40 + item_log2)
    plan = pir.pir_multi_plan_create(dts, assign, item_log2)
    shares = []
    for keys in (ks0, ks1):
        out = torch.full((plan.out_words_total,), -1, dtype=torch.int32, device="cuda")
        pir.pir_server_eval_multi(plan, _pack(torch, plan, keys), out)
        torch.cuda.synchronize()
        got = _unpack(plan, out, SHAPES, assign)
        for q, t in enumerate(assign):
            assert np.array_equal(got[q], orc.answer(keys[q], Ts[t])), (q, t)
        shares.append(got)
    for q, t in enumerate(assign):
        rec = (shares[0][q].astype(np.uint64) + shares[1][q]) & M32
        assert np.array_equal(rec.astype(np.uint32), Ts[t][alphas[q]])


def test_graph_replay_reads_current_keys(env):
    torch, pir, orc = env
    assign = [0, 2, 2, 1, 5, 0, 0, 2, 2, 2, 2, 2, 2, 2, 2, 3]
    Ts, dts, alphas, ks0, ks1 = _mix(torch, pir, orc, SHAPES, assign, 77)
    plan = pir.pir_multi_plan_create(dts, assign)
    dkeys = _pack(torch, plan, ks0)
    out = torch.empty((plan.out_words_total,), dtype=torch.int32, device="cuda")
    graph = pir.pir_multi_graph_create(plan, dkeys, out)
    direct = torch.empty_like(out)
    pir.pir_server_eval_multi(plan, dkeys, direct)
    graph.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, direct)
    dkeys.copy_(_pack(torch, plan, ks1))  # same buffer, new keys: the replay evaluates them
    graph.launch()
    torch.cuda.synchronize()
    got = _unpack(plan, out, SHAPES, assign)
    for q, t in enumerate(assign):
        assert np.array_equal(got[q], orc.answer(ks1[q], Ts[t]))
    graph.close()


def test_autotune_picks_a_working_item_size(env):
    torch, pir, orc = env
    assign = ([0] * 9 + [5] * 3 + [2] * 8)
    Ts, dts, alphas, ks0, _ = _mix(torch, pir, orc, SHAPES, assign, 9)
    plan = pir.pir_multi_plan_create(dts, assign)
    dkeys = _pack(torch, plan, ks0)
    out = torch.empty((plan.out_words_total,), dtype=torch.int32, device="cuda")
    best, ms = pir.pir_multi_autotune(dts, assign, dkeys, out)
    assert 11 <= best <= 15 and ms > 0
    tuned = pir.pir_multi_plan_create(dts, assign, best)
    pir.pir_server_eval_multi(tuned, dkeys, out)
    torch.cuda.synchronize()
    got = _unpack(tuned, out, SHAPES, assign)
    for q in (0, 9, 19):
        assert np.array_equal(got[q], orc.answer(ks0[q], Ts[assign[q]]))


def test_multi_bad_key_sets_status_and_zero_share(env):
    torch, pir, orc = env
    assign = [1, 1, 2, 0]
    Ts, dts, alphas, ks0, _ = _mix(torch, pir, orc, SHAPES, assign, 3)
    bad = bytearray(ks0[2])
    bad[5] = 7  # wrong n for its table
    keys = [ks0[0], ks0[1], bytes(bad), ks0[3]]
    plan = pir.pir_multi_plan_create(dts, assign)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((plan.out_words_total,), dtype=torch.int32, device="cuda")
    pir.pir_server_eval_multi(plan, _pack(torch, plan, keys), out, status)
    torch.cuda.synchronize()
    got = _unpack(plan, out, SHAPES, assign)
    assert int(status.item()) & 1 and not got[2].any()
    for q in (0, 1, 3):
        assert np.array_equal(got[q], orc.answer(keys[q], Ts[assign[q]]))


def test_multi_refuses_widths_its_consumers_cannot_cover(env):
    """A table that is not 16-byte aligned puts the kernel on 32-bit loads, and
    then a row of more than 256 words would be left to no consumer: the
    planner refuses it instead of returning zero shares."""
    torch, pir, _ = env
    wide = torch.zeros((64, 301), dtype=torch.int32, device="cuda")  # 301 words: not a multiple of 4
    narrow = torch.zeros((64, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:
        pir.pir_multi_plan_create([narrow, wide], [0, 1])
    assert e.value.code == -8
    ok = torch.zeros((64, 300), dtype=torch.int32, device="cuda")  # 16-byte rows: 75 chunks of 4 words
    pir.pir_multi_plan_create([narrow, ok], [0, 1]).close()


def test_multi_table_full_size_zipf_mix(env):
    """8 tables, rows 2^16..2^22, widths {16,32,32,64,64,128,32,16} words, 2048
    queries Zipf(1.1) over the table order, in the bench's launch
    configuration: all queries reconstruct T[alpha]; 16 sampled queries per
    table (all of a table's queries when it has fewer) match the oracle's
    per-server share word for word."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    torch, pir, orc = env
    shapes = list(zip(wl.MULTI_TABLE_ROWS, wl.MULTI_TABLE_WIDTHS))
    assign = wl.zipf_assignment(303, len(shapes), wl.MULTI_TABLE_QUERIES).tolist()
    tables = [wl.table_u32_torch(300 + i, r, w, "cuda") for i, (r, w) in enumerate(shapes)]
    rng = np.random.Generator(np.random.PCG64(303))
    alphas = [int(rng.integers(0, shapes[t][0])) for t in assign]
    plan = pir.pir_multi_plan_create(tables, assign)
    ks = ([], [])
    for q, t in enumerate(assign):
        k0, k1 = pir.pir_keygen(pir.pir_domain_bits(shapes[t][0]), alphas[q], 1, bytes([q & 255, q >> 8]) * 16)
        ks[0].append(k0)
        ks[1].append(k1)
    outs = []
    for party in (0, 1):
        out = torch.empty((plan.out_words_total,), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_multi(plan, _pack(torch, plan, ks[party]), out)
        torch.cuda.synchronize()
        outs.append(_unpack(plan, out, shapes, assign))
    for q, t in enumerate(assign):
        rec = (outs[0][q].astype(np.uint64) + outs[1][q]) & M32
        row = tables[t][alphas[q]].cpu().numpy().view(np.uint32)
        assert np.array_equal(rec.astype(np.uint32), row), q
    host = [t.cpu().numpy().view(np.uint32) for t in tables]
    sample = []
    for t in range(len(shapes)):
        qs = [q for q, tt in enumerate(assign) if tt == t]
        sample += qs[:: max(1, len(qs) // 16)][:16]
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        wants = list(ex.map(lambda q: orc.answer(ks[0][q], host[assign[q]]), sample))
    for q, want in zip(sample, wants):
        assert np.array_equal(outs[0][q], want), q
