"""Failure paths that need no GPU fault: a device wait whose bound runs out
(on an mbarrier nothing completes) reports PIR_FAULT_WAIT_TIMEOUT and leaves
the context usable; requests cancelled before they run are withdrawn (their
buffers untouched, their tickets released) while the rest complete exactly."""
import time

import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_table, make_keys

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


def test_bounded_wait_runs_out_and_reports(env):
    torch, pir, orc = env
    pir.pir_device_status(clear=True)
    assert pir.pir_selftest_bounded_wait(4096) == -6  # PIR_ERR_TIMEOUT: the bound ran out
    assert pir.pir_device_status() & pir.PIR_FAULT_WAIT_TIMEOUT
    assert pir.pir_device_status(clear=True) & pir.PIR_FAULT_WAIT_TIMEOUT
    assert pir.pir_device_status() == 0
    # the context is still usable: an evaluation right after is exact
    rows, W = 3000, 8
    T = wl.table_u32(61, rows, W)
    n = pir.pir_domain_bits(rows)
    ks0, _ = make_keys(orc, n, [1234], [1], 61)
    dk = torch.frombuffer(bytearray(ks0[0]), dtype=torch.uint8).cuda()
    out = torch.empty((1, W), dtype=torch.int32, device="cuda")
    pir.pir_server_eval_device(dev_table(torch, T), dk, 1, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], orc.answer(ks0[0], T))


def test_cancel_withdraws_pending_requests(env):
    torch, pir, orc = env
    rows, W = 1 << 22, 32
    table = wl.table_u32_torch(62, rows, W, "cuda")
    n = pir.pir_domain_bits(rows)
    srv = pir.Server(max_batch=1, streams=1)  # one query at a time: the rest wait in the queue
    tid = srv.register_table(table)
    alphas = [11, 22, 33, 44, 55, 66, 77]
    pairs = [pir.pir_keygen(n, a, 1, bytes([i]) * 32) for i, a in enumerate(alphas)]
    outs = [np.full(W, 0xA5A5A5A5, np.uint32) for _ in alphas]
    tickets = [srv.submit(tid, p[0], o) for p, o in zip(pairs, outs)]
    cancelled = [srv.cancel(t) for t in tickets[3:]][::-1]  # newest first: the queue's tail
    assert cancelled[0], "the last of seven queued requests was still waiting"
    n_cancelled = sum(cancelled)
    done = set()
    t0 = time.time()
    while len(done) < len(tickets) - n_cancelled:
        for i, t in enumerate(tickets):
            if i in done or (i >= 3 and cancelled[len(tickets) - 1 - i]):
                continue
            if srv.poll(t) is not None:
                done.add(i)
        assert time.time() - t0 < 60
        time.sleep(0.0005)
    for i, t in enumerate(tickets):
        if i >= 3 and cancelled[len(tickets) - 1 - i]:
            assert (outs[i] == 0xA5A5A5A5).all()  # never written
            with pytest.raises(pir.PirError):
                srv.poll(t)  # the ticket was released
        else:
            # the other party's share, computed alone, reconstructs the row
            other = torch.empty((1, W), dtype=torch.int32, device="cuda")
            pir.pir_server_eval_device(table, torch.frombuffer(bytearray(pairs[i][1]), dtype=torch.uint8).cuda(), 1,
                                       other)
            torch.cuda.synchronize()
            rec = (outs[i].astype(np.uint64) + other.cpu().numpy().view(np.uint32)[0]) & 0xFFFFFFFF
            assert np.array_equal(rec.astype(np.uint32), table[alphas[i]].cpu().numpy().view(np.uint32))
    assert srv.stats()["cancelled"] == n_cancelled
    srv.close()


def test_host_call_reports_only_timeouts_of_its_own_kernels(env):
    """pir_server_eval with a host `out` snapshots the device fault word around
    kernels with bounded waits (here the expand-and-scan strategy of one query
    on 128 MiB of 64-word rows) and returns PIR_ERR_TIMEOUT only for a bit
    that one of them set: a bit left set by an earlier launch (the bounded-wait
    diagnostic) is not this call's, and the call returns the exact shares."""
    torch, pir, orc = env
    rows, W = 1 << 19, 64
    assert pir.pir_plan_for(rows, W, 1).strategy == pir.PIR_STRATEGY_EXPAND_SCAN
    table = wl.table_u32_torch(63, rows, W, "cuda")
    n = pir.pir_domain_bits(rows)
    ks0, ks1 = make_keys(orc, n, [rows - 7], [1], 63)
    pir.pir_device_status(clear=True)
    assert pir.pir_selftest_bounded_wait(4096) == -6  # leaves PIR_FAULT_WAIT_TIMEOUT set
    shares = []
    for k in (ks0[0], ks1[0]):
        out = np.zeros((1, W), np.uint32)
        pir.pir_server_eval(table, k, 1, out)  # raises on PIR_ERR_TIMEOUT
        shares.append(out[0])
    assert pir.pir_device_status(clear=True) & pir.PIR_FAULT_WAIT_TIMEOUT  # still set, not cleared by the call
    T = table.cpu().numpy().view(np.uint32)
    assert np.array_equal(shares[0], orc.answer(ks0[0], T))
    assert np.array_equal(pir.pir_reconstruct(shares[0], shares[1]), T[rows - 7])
