"""Parity of the fused kernel whose table scan is staged through shared memory
(PIR_STRATEGY_FUSED_STAGED): one more warp has the bulk-copy engine move each
hand-off's table rows into a ring of shared-memory stages, and the consumers
multiply them from there.  Every share is compared word for word with the
oracle's T x Eval(k, .) mod 2^32 (Sec. 3.1), on ragged shapes, padded rows,
every launch shape the strategy accepts (query groups, rows per item, cut last
rounds), bad keys, and at the full 2^20 x 64 and 2^24 x 32 sizes against the
other strategies and sampled oracle queries.  No wait of the ring may give up
(the library's device fault word stays clear)."""
import os

import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_keys, dev_table, make_keys, run_device

pytestmark = pytest.mark.gpu
M32 = 0xFFFFFFFF
STAGED = 2


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import oracle
    import paper_2301_10904_gb300 as pir

    pir.pir_device_status(clear=True)
    return torch, pir, oracle


def staged_plan(pir, rows, W, B):
    """The heuristic plan as a staged one: query group at most 4, rows per item
    lowered until the subtrees leave the ring at least two stack levels."""
    plan = pir.pir_plan_for(rows, W, B)
    plan.strategy = STAGED
    plan.vec = 4
    while plan.group > min(4, B):
        plan.group //= 2
    lsq = {1: 9, 2: 8, 4: 7}[plan.group]
    n = pir.pir_domain_bits(rows)
    plan.range_log2 = min(plan.range_log2, n)
    while plan.range_log2 > 1 and plan.range_log2 - min(lsq, plan.range_log2 - 1) > 7:
        plan.range_log2 -= 1
    plan.tail_log2 = min(plan.tail_log2, max(0, plan.range_log2 - 1), 3)
    return plan


SHAPES = [  # (rows, width, batch, pad words per row): several items, ragged tails, padded rows
    (2, 4, 1, 0), (3, 4, 2, 0), (1000, 16, 3, 0), (4096 + 77, 16, 3, 4), (1 << 14, 64, 4, 0),
    ((1 << 15) + 1000, 32, 2, 4), (1 << 13, 100, 4, 0), (1 << 11, 256, 1, 0), (5000, 4, 1, 8),
    (3000, 8, 2, 0), ((1 << 16) + 5, 64, 1, 0), ((1 << 17) - 3, 12, 4, 4),
]


def padded_table(torch, T, pad, seed):
    rows, W = T.shape
    full = np.random.Generator(np.random.PCG64(seed)).integers(0, 1 << 32, (rows, W + pad),
                                                               dtype=np.uint64).astype(np.uint32)
    full[:, :W] = T
    return dev_table(torch, full)[:, :W]


@pytest.mark.parametrize("rows,width,batch,pad", SHAPES)
def test_staged_matches_oracle(env, rows, width, batch, pad):
    torch, pir, orc = env
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(rows * 5 + width, rows, width)
    alphas = wl.alphas(rows + 1, rows, batch)
    alphas[0] = rows - 1
    betas = [1] * batch
    if batch > 1:
        betas[1] = M32
    ks0, ks1 = make_keys(orc, n, alphas, betas, rows + 3 * batch)
    table = padded_table(torch, T, pad, rows + 9) if pad else dev_table(torch, T)
    plan = staged_plan(pir, rows, width, batch)
    g0 = run_device(torch, pir, table, ks0, width, plan=plan)
    g1 = run_device(torch, pir, table, ks1, width, plan=plan)
    for q in range(batch):
        assert np.array_equal(g0[q], orc.answer(ks0[q], T)), (q, plan.as_dict())
        assert np.array_equal(g1[q], orc.answer(ks1[q], T)), (q, plan.as_dict())
        want = (T[alphas[q]].astype(np.uint64) * betas[q]) & M32
        assert np.array_equal(pir.pir_reconstruct(g0[q], g1[q]), want.astype(np.uint32))
    assert pir.pir_device_status(clear=True) == 0


def test_every_staged_launch_shape_matches_oracle(env):
    # every (group, rows per item, cut of the last round) the strategy accepts
    torch, pir, orc = env
    rows, width, batch = (1 << 14) + 333, 32, 5
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(23, rows, width)
    alphas = wl.alphas(4, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, 78)
    want = np.stack([orc.answer(k, T) for k in ks0])
    table = dev_table(torch, T)
    ran = refused = 0
    for g in (1, 2, 4):
        for r in range(1, n + 1):
            for tail in (0, 2):
                if tail > r - 1:
                    continue
                plan = pir.pir_plan(g, r, 4, 0, STAGED, tail)
                try:
                    got = run_device(torch, pir, table, ks0, width, plan=plan)
                except pir.PirError as e:
                    assert e.code == -8, plan.as_dict()  # subtrees too deep for a ring
                    refused += 1
                    continue
                assert np.array_equal(got, want), plan.as_dict()
                ran += 1
    assert ran >= 60 and refused > 0
    assert pir.pir_device_status(clear=True) == 0


def test_staged_refuses_what_it_cannot_stage(env):
    torch, pir, orc = env
    rows, width = 4096, 16
    T = wl.table_u32(5, rows, width)
    ks0, _ = make_keys(orc, pir.pir_domain_bits(rows), [7], [1], 6)
    table = dev_table(torch, T)
    for plan in (pir.pir_plan(8, 9, 4, 0, STAGED, 0),   # eight queries per item
                 pir.pir_plan(1, 9, 1, 0, STAGED, 0)):  # 32-bit loads
        with pytest.raises(pir.PirError) as e:
            run_device(torch, pir, table, ks0, width, plan=plan)
        assert e.value.code == -8
    wide = dev_table(torch, wl.table_u32(6, 512, 260))  # rows wider than a quarter stage
    with pytest.raises(pir.PirError) as e:
        run_device(torch, pir, wide, make_keys(orc, 9, [3], [1], 7)[0], 260, plan=pir.pir_plan(1, 9, 4, 0, STAGED, 0))
    assert e.value.code == -8


def test_staged_bad_key_gives_zero_share_and_status(env):
    torch, pir, orc = env
    rows, W = 1 << 14, 32
    T = wl.table_u32(8, rows, W)
    n = pir.pir_domain_bits(rows)
    ks0, _ = make_keys(orc, n, [5, 9000], [1, 1], 9)
    bad = bytearray(ks0[0])
    bad[5] = n - 1  # wrong domain
    keys = [bytes(bad), ks0[1]]
    table = dev_table(torch, T)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = run_device(torch, pir, table, keys, W, plan=staged_plan(pir, rows, W, 2), status=status)
    assert not got[0].any() and int(status.item()) & pir.PIR_STATUS_BAD_KEY
    assert np.array_equal(got[1], orc.answer(ks0[1], T))


def _oracle_many(orc, keys, T):
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max(1, min(len(keys), os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda k: orc.answer(k, T), keys))


@pytest.mark.parametrize("batch", [1, 2, 4])
def test_staged_full_size_2p20x64(env, batch):
    """The 256 MiB table with 1, 2 and 4 queries: staged shares equal the fused
    kernel's and the expand-and-scan strategy's word for word, every query's
    equals the oracle's, and both servers reconstruct T[alpha]."""
    torch, pir, orc = env
    rows, W = 1 << 20, 64
    n = pir.pir_domain_bits(rows)
    table = wl.table_u32_torch(202, rows, W, "cuda")
    alphas = wl.alphas(210 + batch, rows, batch)
    alphas[0] = rows - 1
    ks0, ks1 = make_keys(orc, n, alphas, [1] * batch, 220 + batch)
    plan = staged_plan(pir, rows, W, batch)
    got = run_device(torch, pir, table, ks0, W, plan=plan)
    got1 = run_device(torch, pir, table, ks1, W, plan=plan)
    for strategy in (0, 1):
        other = pir.pir_plan_for(rows, W, batch)
        other.strategy = strategy
        assert np.array_equal(run_device(torch, pir, table, ks0, W, plan=other), got), strategy
    T = table.cpu().numpy().view(np.uint32)
    for q, want in enumerate(_oracle_many(orc, ks0, T)):
        assert np.array_equal(got[q], want), q
    rec = ((got.astype(np.uint64) + got1) & M32).astype(np.uint32)
    assert np.array_equal(rec, T[alphas])
    assert pir.pir_device_status(clear=True) == 0


def test_staged_full_size_2p24x32_one_query(env):
    """One query on the 2 GiB table: the staged share equals the oracle's (both
    servers) and the fused kernel's, and reconstructs T[alpha]."""
    torch, pir, orc = env
    rows, W = 1 << 24, 32
    n = pir.pir_domain_bits(rows)
    table = wl.table_u32_torch(404, rows, W, "cuda")
    alpha = 12_345_678
    ks0, ks1 = make_keys(orc, n, [alpha], [1], 405)
    plan = staged_plan(pir, rows, W, 1)
    g0 = run_device(torch, pir, table, ks0, W, plan=plan)[0]
    g1 = run_device(torch, pir, table, ks1, W, plan=plan)[0]
    fused = pir.pir_plan_for(rows, W, 1)
    fused.strategy = 0
    assert np.array_equal(run_device(torch, pir, table, ks0, W, plan=fused)[0], g0)
    T = table.cpu().numpy().view(np.uint32)
    w0, w1 = _oracle_many(orc, [ks0[0], ks1[0]], T)
    assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
    assert np.array_equal(pir.pir_reconstruct(g0, g1), T[alpha])
    assert pir.pir_device_status(clear=True) == 0


def test_staged_strategy_through_the_host_entry_point(env):
    """A staged plan pinned for the shape runs through pir_server_eval's
    graph (keys in, the staged kernel between two snapshots of the device
    fault word, shares out): calls with new keys on the same graph give the
    oracle's shares, and a fault bit left set before the calls (by the
    bounded-wait diagnostic) is not reported as theirs."""
    torch, pir, orc = env
    rows, W, batch = (1 << 15) + 1000, 32, 2
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(91, rows, W)
    table = dev_table(torch, T)
    plan = staged_plan(pir, rows, W, batch)
    pir.pir_plan_pin(table, batch, plan)
    try:
        assert pir.pir_plan_for(rows, W, batch).strategy == STAGED
        pir.pir_device_status(clear=True)
        assert pir.pir_selftest_bounded_wait(4096) == -6  # leaves PIR_FAULT_WAIT_TIMEOUT set
        for i in range(3):
            ks0, ks1 = make_keys(orc, n, wl.alphas(500 + i, rows, batch), [1] * batch, 600 + i)
            out0 = np.full((batch, W), 0x5A5A5A5A, np.uint32)
            out1 = np.full((batch, W), 0x5A5A5A5A, np.uint32)
            pir.pir_server_eval(table, b"".join(ks0), batch, out0)  # raises on PIR_ERR_TIMEOUT
            pir.pir_server_eval(table, b"".join(ks1), batch, out1)
            for q in range(batch):
                assert np.array_equal(out0[q], orc.answer(ks0[q], T)), (i, q)
                assert np.array_equal(out1[q], orc.answer(ks1[q], T)), (i, q)
        assert pir.pir_device_status(clear=True) == pir.PIR_FAULT_WAIT_TIMEOUT  # the diagnostic's bit only
    finally:
        pir.pir_plan_pin(table, batch, None)
