"""Frequency-based hot/full table split (Sec. 4) on the host: the oracle's
request plan against worked examples, and the library's client side
(pir_hotfull_keygen) against the oracle, with every kept row reconstructed
from both tables' answers and every dummy query answering zero.  No GPU."""
import numpy as np
import pytest

import workloads as wl

M32 = 0xFFFFFFFF


@pytest.fixture(scope="module")
def pir():
    import __graft_entry__ as g

    g.build_library()
    import paper_2301_10904_gb300 as pir

    return pir


def test_hotfull_plan_worked_example(orc):
    hot_rows = [3, 10, 40]  # hot row h holds full row hot_rows[h]
    # 10 and 3 are hot: hot queries 0 and 1; 7 is not: full query 0; 40 is hot but
    # the hot budget (2) is spent: full query 1; 11 finds both budgets spent: dropped
    ha, hb, fa, fb, slots = orc.hotfull_plan(64, hot_rows, [10, 3, 7, 40, 11], q_hot=2, q_full=2)
    assert (ha, hb) == ([1, 0], [1, 1])
    assert (fa, fb) == ([7, 40], [1, 1])
    assert slots == [0, 1, 2, 3, -1]
    # a light request: unused queries are dummies
    ha, hb, fa, fb, slots = orc.hotfull_plan(64, hot_rows, [40], q_hot=2, q_full=3)
    assert (ha, hb, fa, fb, slots) == ([2, 0], [1, 0], [0, 0, 0], [0, 0, 0], [0])


@pytest.mark.parametrize("q_hot,q_full", [(4, 2), (1, 0), (0, 3), (8, 8)])
def test_library_hotfull_keys_follow_the_oracle_plan(pir, orc, q_hot, q_full):
    full_rows, W = 3000, 4
    rng = np.random.Generator(np.random.PCG64(q_hot * 10 + q_full))
    hot_rows = np.sort(rng.choice(full_rows, 300, replace=False))
    T = wl.table_u32(11, full_rows, W)
    H = T[hot_rows]
    wanted = [int(hot_rows[5]), 17, int(hot_rows[9]), int(hot_rows[5]), 2999, 1, int(hot_rows[0])]
    hk0, hk1, fk0, fk1, slot = pir.pir_hotfull_keygen(full_rows, hot_rows, wanted, q_hot, q_full,
                                                      seed=b"\x03" * 32)
    ha, hb, fa, fb, want_slots = orc.hotfull_plan(full_rows, hot_rows, wanted, q_hot, q_full)
    assert slot.tolist() == want_slots
    nh, nf = pir.pir_domain_bits(len(hot_rows)), pir.pir_domain_bits(full_rows)
    hkb, fkb = pir.pir_key_bytes(nh), pir.pir_key_bytes(nf)
    assert len(hk0) == q_hot * hkb and len(fk0) == q_full * fkb
    rec = []
    for s in range(q_hot):
        r = (orc.answer(hk0[s * hkb:(s + 1) * hkb], H).astype(np.uint64) + orc.answer(hk1[s * hkb:(s + 1) * hkb], H))
        rec.append(r & M32)
        assert np.array_equal(rec[-1], H[ha[s]] if hb[s] else np.zeros(W, np.uint64))
    for s in range(q_full):
        r = (orc.answer(fk0[s * fkb:(s + 1) * fkb], T).astype(np.uint64) + orc.answer(fk1[s * fkb:(s + 1) * fkb], T))
        rec.append(r & M32)
        assert np.array_equal(rec[-1], T[fa[s]] if fb[s] else np.zeros(W, np.uint64))
    for i, idx in enumerate(wanted):
        if slot[i] >= 0:
            assert np.array_equal(rec[slot[i]], T[idx])


def test_hotfull_errors(pir):
    with pytest.raises(pir.PirError):  # hot rows not increasing
        pir.pir_hotfull_keygen(100, [5, 3], [1], 1, 1)
    with pytest.raises(pir.PirError):  # wanted row past the table
        pir.pir_hotfull_keygen(100, [3, 5], [100], 1, 1)
    with pytest.raises(pir.PirError):  # hot row past the table
        pir.pir_hotfull_keygen(100, [3, 100], [1], 1, 1)
