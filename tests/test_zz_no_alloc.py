"""The allocation-free server entry point (pir_server_eval_noalloc).

Some callers cannot let the library allocate device memory (a host runtime
that owns the whole device budget, or a request path that must not touch the
allocator).  This entry point stages keys and shares through a fixed region
inside the library image instead.  The test calls it through the C ABI twice
in a row, with different keys and shapes, and checks each result against the
allocating entry point pir_server_eval (bit-exact: all arithmetic is integer
mod 2^32), so a stale staging region from the first call would show up in the
second.  This file is collected last on purpose.
"""
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
    import paper_2301_10904_gb300 as pir

    return torch, pir


def _case(torch, pir, rows, width, batch, seed):
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(seed, rows, width)
    table = torch.from_numpy(T.view(np.int32)).cuda()
    alphas = wl.alphas(seed, rows, batch)
    pairs = [pir.pir_keygen(n, int(a), 1, bytes([seed, q]) * 16) for q, a in enumerate(alphas)]
    return T, table, alphas, pairs


def test_noalloc_matches_allocating_entry_point_twice(env):
    torch, pir = env
    results = []
    for rows, width, batch, seed in ((5000, 16, 7, 1), (1 << 12, 64, 3, 2)):
        T, table, alphas, pairs = _case(torch, pir, rows, width, batch, seed)
        shares = []
        for party in (0, 1):
            keys = b"".join(p[party] for p in pairs)
            want = np.zeros((batch, width), np.uint32)
            pir.pir_server_eval(table, keys, batch, want)
            got = np.full((batch, width), 0xDEADBEEF, np.uint32)
            pir.pir_server_eval_noalloc(table, keys, batch, got)
            assert np.array_equal(got, want)
            shares.append(got)
        rec = (shares[0].astype(np.uint64) + shares[1]) & 0xFFFFFFFF
        assert np.array_equal(rec.astype(np.uint32), T[alphas])
        results.append(rec)
    assert len(results) == 2


def test_noalloc_rejects_batches_beyond_its_region(env):
    torch, pir = env
    T, table, _, pairs = _case(torch, pir, 1 << 12, 64, 1, 3)
    kb = pir.pir_key_bytes(12)
    too_many = (192 * 1024) // kb + 1
    keys = pairs[0][0] * too_many
    out = np.zeros((too_many, 64), np.uint32)
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval_noalloc(table, keys, too_many, out)
    assert e.value.code == -8


def test_noalloc_allocates_no_device_memory(env):
    """After one warm-up call (the region's one-time address lookup), calls of
    several shapes leave the device's free memory and the library's staging
    pool (reserved and in-use bytes) exactly as they were."""
    torch, pir = env
    cases = [_case(torch, pir, rows, width, batch, seed)
             for rows, width, batch, seed in ((5000, 16, 7, 4), (1 << 12, 64, 3, 5), (1 << 14, 8, 20, 6))]
    T, table, alphas, pairs = cases[0]
    out = np.zeros((len(pairs), T.shape[1]), np.uint32)
    pir.pir_server_eval_noalloc(table, b"".join(p[0] for p in pairs), len(pairs), out)
    torch.cuda.synchronize()
    free0, pool0 = torch.cuda.mem_get_info()[0], pir.pir_staging_stats()
    for _ in range(3):
        for T, table, alphas, pairs in cases:
            got = np.zeros((len(pairs), T.shape[1]), np.uint32)
            pir.pir_server_eval_noalloc(table, b"".join(p[0] for p in pairs), len(pairs), got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert pir.pir_staging_stats() == pool0


def test_noalloc_refuses_a_device_output(env):
    """The shares are copied back to host memory: a device `out` is an
    argument error, not a copy into device memory."""
    torch, pir = env
    T, table, _, pairs = _case(torch, pir, 5000, 16, 2, 7)
    dout = torch.zeros((2, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval_noalloc(table, b"".join(p[0] for p in pairs), 2, dout)
    assert e.value.code == -1
    assert not dout.any()
