"""The multi-table planner's host logic (pir_multi_plan_inspect, no device):
every query of a table is covered once per row range of that table, a range's
items are adjacent, query slots come in powers of two with full groups of 8,
rows per item follow item_log2 (or the cost model's bounds when it is 0), and
widths the kernel's consumers cannot cover are refused."""
import collections

import pytest


@pytest.fixture(scope="module")
def pir():
    import __graft_entry__ as g

    g.build_library()
    import paper_2301_10904_gb300 as pir

    return pir


def _domain_bits(rows):
    return max(1, (rows - 1).bit_length())


def _check_cover(items, tables, table_of_key):
    per_table = collections.defaultdict(list)
    for q, t in enumerate(table_of_key):
        per_table[t].append(q)
    seen = collections.defaultdict(list)  # (table, range) -> queries
    order = []
    for it in items:
        key = (it["table"], it["range"])
        if not order or order[-1] != key:
            assert key not in order, "a range's items are not adjacent"
            order.append(key)
        g = it["group"]
        assert g in (1, 2, 4, 8) and 1 <= len(it["queries"]) <= g
        assert len(it["queries"]) > g // 2 or g == 1  # the smallest power of two that holds them
        seen[key] += it["queries"]
    for t, qs in per_table.items():
        rows = tables[t][0]
        r = next(it["range_log2"] for it in items if it["table"] == t)
        ranges = ((rows - 1) >> r) + 1
        for rg in range(ranges):
            assert sorted(seen[(t, rg)]) == qs  # each query once per range
    assert set(k[0] for k in seen) == set(per_table)


@pytest.mark.parametrize("counts", [[1, 1, 1], [8, 3, 17], [0, 5, 9], [64, 0, 1]])
def test_items_cover_every_query_once_per_range(pir, counts):
    tables = [(1 << 16, 16), (5000, 32), ((1 << 20) + 7, 64)]
    table_of_key = [t for t, c in enumerate(counts) for _ in range(c)]
    items = pir.pir_multi_plan_inspect(tables, table_of_key, item_log2=12)
    _check_cover(items, tables, table_of_key)
    for it in items:
        assert it["range_log2"] == min(_domain_bits(tables[it["table"]][0]), 12)
    # full groups of 8, then one smaller power-of-two group
    for t, c in enumerate(counts):
        groups = [it["group"] for it in items if it["table"] == t and it["range"] == 0]
        if c:
            assert groups[:-1] == [8] * (len(groups) - 1) and sum(len(it["queries"]) for it in items
                                                                    if it["table"] == t and it["range"] == 0) == c


def test_automatic_rows_per_item_respect_the_subtree_bound(pir):
    tables = [(1 << 24, 16), (1 << 20, 32)]
    lone = pir.pir_multi_plan_inspect(tables, [0], item_log2=0)
    # one query: one slot per item, whose 512 producers' subtrees may be 9 levels deep
    assert {it["group"] for it in lone} == {1}
    assert 10 <= lone[0]["range_log2"] <= 18
    _check_cover(lone, tables, [0])
    many = pir.pir_multi_plan_inspect(tables, [0] * 20 + [1] * 3, item_log2=0)
    _check_cover(many, tables, [0] * 20 + [1] * 3)
    for it in many:
        bound = {8: 15, 4: 16, 2: 17, 1: 18}[max(x["group"] for x in many if x["table"] == it["table"])]
        assert it["range_log2"] <= bound


def test_widths_beyond_the_consumers_are_refused(pir):
    with pytest.raises(pir.PirError) as e:  # not 16-byte aligned: 32-bit loads, 301 chunks > 256
        pir.pir_multi_plan_inspect([(64, 8), (64, 301, 301, False)], [0, 1])
    assert e.value.code == -8
    assert pir.pir_multi_plan_inspect([(64, 8), (64, 300)], [0, 1])  # 75 chunks of 4 words
    with pytest.raises(pir.PirError):
        pir.pir_multi_plan_inspect([(64, 8)], [1])  # no table 1
