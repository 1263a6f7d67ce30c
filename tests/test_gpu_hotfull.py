"""Hot/full table split (Sec. 4) end to end on the GPU: requests planned by
pir_hotfull_keygen, served through the serving loop over the hot and the full
table (both parties), every kept row reconstructed and every dummy query
answering zero; one request's shares also against the oracle."""
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


def test_hotfull_requests_through_the_serving_loop(env):
    torch, pir, orc = env
    full_rows, W, hot_n, K, qh, qf = 1 << 14, 16, 1 << 10, 6, 4, 2
    q = qh + qf
    z = wl.ZipfRows(3, full_rows)
    hot_rows = z.top(hot_n)
    T = wl.table_u32(4, full_rows, W)
    full = torch.from_numpy(T.view(np.int32)).cuda()
    hot = full[torch.from_numpy(hot_rows.astype(np.int64)).cuda()].contiguous()
    srv = pir.Server(max_batch=256, streams=2)
    th, tf = srv.register_table(hot), srv.register_table(full)
    R = 40
    wanted = z.sample(5, R * K).reshape(R, K)
    shares = []
    slots = []
    keys_first = None
    for party in (0, 1):
        ks, tids = [], []
        for r in range(R):
            hk0, hk1, fk0, fk1, slot = pir.pir_hotfull_keygen(full_rows, hot_rows, wanted[r], qh, qf,
                                                              seed=bytes([r]) * 32)
            hk, fk = (hk0, fk0) if party == 0 else (hk1, fk1)
            hkb, fkb = len(hk) // qh, len(fk) // qf
            ks += [hk[i * hkb:(i + 1) * hkb] for i in range(qh)] + [fk[i * fkb:(i + 1) * fkb] for i in range(qf)]
            tids += [th] * qh + [tf] * qf
            if party == 0:
                slots.append(slot)
                if r == 0:
                    keys_first = (hk0[:hkb], fk0[:fkb])
        koff = np.concatenate([[0], np.cumsum([len(k) for k in ks])[:-1]]).astype(np.uint64)
        outs = np.zeros(R * q * W, np.uint32)
        arr = np.repeat(np.arange(R) * 1e-4, q)
        srv.replay(arr, tids, b"".join(ks), koff, outs, np.arange(R * q, dtype=np.uint64) * W)
        shares.append(outs.reshape(R, q, W))
    srv.close()
    rec = ((shares[0].astype(np.uint64) + shares[1]) & M32).astype(np.uint32)
    kept = 0
    for r in range(R):
        used = set()
        for i, sl in enumerate(slots[r]):
            if sl >= 0:
                assert np.array_equal(rec[r, sl], T[int(wanted[r, i])])
                used.add(int(sl))
                kept += 1
        for sl in set(range(q)) - used:
            assert not rec[r, sl].any()  # dummy query
    assert kept >= R * min(K, q) * 0.9
    # request 0: the first hot and the first full query against the oracle
    H = T[hot_rows.astype(np.int64)]
    assert np.array_equal(shares[0][0, 0], orc.answer(keys_first[0], H))
    assert np.array_equal(shares[0][0, qh], orc.answer(keys_first[1], T))
