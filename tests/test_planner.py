"""The single-table planner on the host (pir_plan_inspect, no GPU): the plans
of the bench shapes on a 152-SM GB300, the planner's invariants, and its
choice of rows per item and last-round pieces against a restatement of its
cost model, minimised by brute force over every choice."""
import math

import pytest

K_LEVEL_NODES = 130  # one dependent level's latency in node-work units
K_MAX_TAIL_LOG2 = 3
K_MAX_DFS_DEPTH = 9
K_PRODUCERS = 512


@pytest.fixture(scope="module")
def pir():
    import __graft_entry__ as g

    g.build_library()
    import paper_2301_10904_gb300 as pir

    return pir


def _cost(items, sms, n, g, r, s):
    """Makespan in node-work units: whole rounds of whole items, then the last
    round's items cut into 2^s pieces spread over the grid."""
    if items == 0:
        return 0
    c = min(items, sms)
    lat = n * K_LEVEL_NODES
    if s == 0:
        return -(-items // c) * (lat + g * 2 ** r)
    whole = items // c
    cut = items - whole * c
    return whole * (lat + g * 2 ** r) + -(-(cut << s) // c) * (lat + g * 2 ** (r - s))


def _best(rows, width, batch, sms):
    """Every (r, s) the planner may choose; the minimum-cost one, ties to the larger r, then the smaller s."""
    n = max(1, math.ceil(math.log2(rows)))
    g = 8
    while g > 1 and g > batch:
        g >>= 1
    nqg = -(-batch // g)
    r_max = min(n, int(math.log2(K_PRODUCERS // g)) + K_MAX_DFS_DEPTH)
    best = None
    for r in range(r_max, 0, -1):
        items = -(-rows // 2 ** r) * nqg
        for s in range(0, min(K_MAX_TAIL_LOG2, r - 1) + 1):
            key = (_cost(items, sms, n, g, r, s), -r, s)
            if best is None or key < best[0]:
                best = (key, g, r, s, min(items, sms))
    return best[1:]


def test_bench_shapes_on_gb300(pir):
    def shape(rows, width, batch):
        p = pir.pir_plan_inspect(rows, width, batch, 152)
        return p.group, p.range_log2, p.tail_log2, p.ctas, p.vec, p.strategy

    assert shape(1 << 20, 64, 256) == (8, 15, 2, 152, 4, 0)        # batched: 1,024 items, last round cut in 4
    assert shape(1 << 24, 32, 1024) == (8, 15, 2, 152, 4, 0)       # large
    assert shape(1 << 16, 16, 1) == (1, 9, 0, 128, 4, 0)           # one query on 2^16 x 16: fused
    assert shape((1 << 14) + 77, 16, 200) == (8, 11, 1, 152, 4, 0)
    assert shape(1 << 20, 64, 1)[5] == 1                           # a lone query on 256 MiB: expand + scan
    assert shape(1 << 19, 64, 1)[5] == 1                           # 128 MiB of 64-word rows: expand + scan
    assert shape(1 << 20, 128, 2)[5] == 1                          # two queries, 128-word rows: expand + scan
    assert shape(1 << 20, 64, 2)[5] == 0                           # two queries, 64-word rows: fused
    assert shape(1 << 24, 32, 1)[5] == 0                           # 32-word rows: fused, even at 2 GiB
    assert shape(1 << 16, 256, 1)[5] == 0                          # wide rows, 64 MiB table: fused
    assert shape(1 << 20, 63, 1)[4:] == (1, 0)                     # unaligned rows: 32-bit loads, fused


@pytest.mark.parametrize("sms", [1, 8, 100, 152])
def test_choice_minimises_the_cost_model(pir, sms):
    checked = 0
    for rows in (2, 3, 100, 1000, 4096 + 77, 1 << 14, (1 << 17) + 5, 1 << 20, 1 << 24):
        for batch in (1, 2, 3, 8, 9, 64, 200, 256, 1024):
            for width in (16, 64):
                p = pir.pir_plan_inspect(rows, width, batch, sms)
                g, r, s, ctas = _best(rows, width, batch, sms)
                assert (p.group, p.range_log2, p.tail_log2, p.ctas) == (g, r, s, ctas), (rows, batch, width, sms)
                n = max(1, math.ceil(math.log2(rows)))
                assert 1 <= p.range_log2 <= n and p.tail_log2 <= min(3, p.range_log2 - 1)
                assert p.group <= max(1, batch) and p.group in (1, 2, 4, 8)
                checked += 1
    assert checked == 162


def test_inspect_rejects_bad_arguments(pir):
    for args in ((0, 16, 1, 152), (100, 0, 1, 152), (100, 16, 0, 152), (100, 16, 1, 0)):
        with pytest.raises(pir.PirError) as e:
            pir.pir_plan_inspect(*args)
        assert e.value.code == -1, args


def test_pinned_plan_is_answered_per_batch_bucket_and_removed(pir):
    """pir_plan_pin stores a checked plan where the autotuner stores its winner
    (batch rounded up to a power of two): pir_plan_for answers it for every
    batch of that bucket, not for the next bucket, and the heuristic's answer
    returns once the entry is removed.  A plan outside the kernels' limits is
    refused.  Host only: the table descriptor is never dereferenced."""
    rows, width = 1 << 16, 64
    t = pir.pir_table(0x100000, rows, width, width)  # a 16-byte-aligned descriptor, no memory behind it
    before = {b: pir.pir_plan_for(rows, width, b).as_dict() for b in (3, 4, 5)}
    pin = pir.pir_plan(2, 10, 4, 0, pir.PIR_STRATEGY_FUSED, 0)
    pir.pir_plan_pin(t, 3, pin)
    try:
        for b in (3, 4):
            got = pir.pir_plan_for(rows, width, b)
            assert (got.group, got.range_log2, got.vec, got.strategy) == (2, 10, 4, pir.PIR_STRATEGY_FUSED)
        assert pir.pir_plan_for(rows, width, 5).as_dict() == before[5]
        staged = pir.pir_plan(2, 9, 4, 0, pir.PIR_STRATEGY_FUSED_STAGED, 0)
        pir.pir_plan_pin(t, 4, staged)  # same bucket: replaces the entry
        assert pir.pir_plan_for(rows, width, 3).strategy == pir.PIR_STRATEGY_FUSED_STAGED
        with pytest.raises(pir.PirError) as e:
            pir.pir_plan_pin(t, 3, pir.pir_plan(2, 17, 4, 0, pir.PIR_STRATEGY_FUSED, 0))  # 2^17 rows per item > 2^16
        assert e.value.code in (-1, -8)
        assert pir.pir_plan_for(rows, width, 3).strategy == pir.PIR_STRATEGY_FUSED_STAGED  # left as it was
    finally:
        pir.pir_plan_pin(t, 3, None)
    assert {b: pir.pir_plan_for(rows, width, b).as_dict() for b in (3, 4, 5)} == before
