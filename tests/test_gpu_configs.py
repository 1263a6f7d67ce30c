"""Parity at the full workload sizes, in the launch configuration bench.py uses
(the library's default plan through pir_server_eval_device).

 - plain single query: 2^16 rows x 16 words, one key pair, both servers,
   every output word against the oracle, then reconstruction;
 - batched: 2^20 rows x 64 words, 256 queries: every query reconstructs
   T[alpha] exactly (both servers on the GPU), every query's server-0 share
   and a seeded sample of 16 server-1 shares match the oracle word for word;
 - large table: 2^24 rows x 32 words (2 GiB), 1024 queries: every query
   reconstructs T[alpha]; 16 seeded server-0 shares (queries 0 and 1023, and
   two more whose last row range runs in the cut last round of the persistent
   grid) and 4 server-1 shares match the oracle word for word.  Reconstruction
   alone would not catch a dropped or misrouted row away from alpha: the two
   servers' shares of such a row are equal and cancel.  The oracle needs tens
   of seconds per 2^24 expansion; the samples run in parallel host threads.
"""
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


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


def _keys(orc, n, alphas, seed):
    ks0, ks1 = [], []
    for (r0, r1, c0), a in zip(wl.key_randomness(seed, n, len(alphas)), alphas):
        k0, k1 = orc.gen(n, int(a), 1, r0, r1, c0)
        ks0.append(k0)
        ks1.append(k1)
    return ks0, ks1


def _eval(torch, pir, table, keys, W):
    dk = torch.frombuffer(bytearray(b"".join(keys)), dtype=torch.uint8).cuda()
    out = torch.empty((len(keys), W), dtype=torch.int32, device="cuda")
    pir.pir_server_eval_device(table, dk, len(keys), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _oracle_sample(orc, keys, T, idx):
    # oracle answers for a few queries, in parallel host threads (ctypes drops the GIL)
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max(1, min(len(idx), os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda q: orc.answer(keys[q], T), idx))


def _check_config(env, rows, width, batch, seed, sample, sample1=None):
    torch, pir, orc = env
    q1 = sample1 if sample1 is not None else sample
    n = pir.pir_domain_bits(rows)
    table = wl.table_u32_torch(seed, rows, width, "cuda")
    alphas = wl.alphas(seed, rows, batch)
    alphas[0] = rows - 1
    alphas[-1] = 0
    ks0, ks1 = _keys(orc, n, alphas, seed)
    g0 = _eval(torch, pir, table, ks0, width)
    g1 = _eval(torch, pir, table, ks1, width)
    rec = (g0.astype(np.uint64) + g1) & 0xFFFFFFFF
    rows_at = table[torch.from_numpy(alphas.astype(np.int64)).cuda()].cpu().numpy().view(np.uint32)
    assert np.array_equal(rec.astype(np.uint32), rows_at)
    T = table.cpu().numpy().view(np.uint32)
    assert np.array_equal(T[[0, rows - 1]], wl.table_rows_u32(seed, width, [0, rows - 1]))
    # both parties' samples in one pool of host threads
    jobs = [(0, q) for q in sample] + [(1, q) for q in q1]
    wants = _oracle_sample(orc, [(ks0, ks1)[s][q] for s, q in jobs], T, range(len(jobs)))
    for (s, q), want in zip(jobs, wants):
        assert np.array_equal((g0, g1)[s][q], want), (s, q)


def test_plain_single_query_2p16x16(env):
    _check_config(env, 1 << 16, 16, 1, 101, [0])


def test_batched_2p20x64_b256(env):
    rng = np.random.Generator(np.random.PCG64(202))
    sample1 = [0, 255] + sorted(set(rng.integers(1, 255, 40).tolist()) - {0, 255})[:14]
    _check_config(env, 1 << 20, 64, 256, 202, list(range(256)), sample1)


def _cut_round_queries(pir, rows, width, batch, sms):
    """Queries whose items run in the persistent grid's cut last round: the
    items past the last whole round of `sms` CTAs, query groups fastest."""
    plan = pir.pir_plan_inspect(rows, width, batch, sms)
    nqg = -(-batch // plan.group)
    nitems = (rows >> plan.range_log2) * nqg
    if not plan.tail_log2:
        return []
    first = nitems // plan.ctas * plan.ctas
    return sorted({(it % nqg) * plan.group + g for it in range(first, nitems) for g in range(plan.group)
                   if (it % nqg) * plan.group + g < batch})


def test_large_2p24x32_b1024(env):
    torch, pir, _ = env
    rows, width, batch = 1 << 24, 32, 1024
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cut = _cut_round_queries(pir, rows, width, batch, sms)
    assert len(cut) >= 3 and 1023 in cut  # the default plan on this device cuts its last round
    rng = np.random.Generator(np.random.PCG64(404))
    pick = [1023, 0] + [int(q) for q in rng.choice([q for q in cut if q != 1023], 2, replace=False)]
    rest = [int(q) for q in rng.permutation(np.arange(1, 1023)) if q not in pick][:16 - len(pick)]
    sample = pick + rest
    assert len(set(sample)) == 16
    _check_config(env, rows, width, batch, 404, sample, [1023, 0] + rest[:2])


def test_single_query_on_a_large_table_two_pass_strategy(env):
    """One query on the 2^20 x 64-word table (256 MiB): the library expands the
    share vector into scratch and streams the table through the scan engine.
    Both parties' shares equal the fused kernel's (explicit plan) word for
    word, one equals the oracle's, the pair reconstructs T[alpha], and a bad
    key gives a zero share and the status bit."""
    torch, pir, orc = env
    rows, W = 1 << 20, 64
    T = wl.table_u32(20, rows, W)
    table = torch.from_numpy(T.view(np.int32)).cuda()
    n = pir.pir_domain_bits(rows)
    alpha = 777_777
    ks0, ks1 = _keys(orc, n, [alpha], 31)
    got = [_eval(torch, pir, table, ks, W)[0] for ks in (ks0, ks1)]
    plan = pir.pir_plan_for(rows, W, 1)
    for ks, g in zip((ks0, ks1), got):
        dk = torch.frombuffer(bytearray(ks[0]), dtype=torch.uint8).cuda()
        fused = torch.empty((1, W), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_device_plan(table, dk, 1, fused, plan)
        torch.cuda.synchronize()
        assert np.array_equal(fused.cpu().numpy().view(np.uint32)[0], g)
    assert np.array_equal(got[0], orc.answer(ks0[0], T))
    rec = ((got[0].astype(np.uint64) + got[1]) & 0xFFFFFFFF).astype(np.uint32)
    assert np.array_equal(rec, T[alpha])
    bad = bytearray(ks0[0])
    bad[5] = 3  # wrong n
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((1, W), 9, dtype=torch.int32, device="cuda")
    pir.pir_server_eval_device(table, torch.frombuffer(bad, dtype=torch.uint8).cuda(), 1, out, status)
    torch.cuda.synchronize()
    assert not out.any() and int(status.item()) & pir.PIR_STATUS_BAD_KEY
