"""The nested (lexicographically sorted) table generator and the counter-based
per-row generator it shares with the device-side generator."""
import numpy as np

from paper_2506_10092_gb300 import datagen as dg


def test_splitmix64_matches_published_outputs():
    # the first outputs of SplitMix64 started from state 0 (Steele, Lea and
    # Flood 2014; the same sequence as Vigna's splitmix64.c seeded with 0)
    got = [int(x) for x in dg.splitmix64(0, 0, np.arange(4))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_is_a_function_of_seed_column_and_row():
    rows = np.array([0, 5, 1 << 40], dtype=np.uint64)
    a = dg.splitmix64(7, 3, rows)
    assert np.array_equal(a, dg.splitmix64(7, 3, rows))
    assert np.array_equal(a[1:2], dg.splitmix64(7, 3, rows[1:2]))
    assert not np.array_equal(a, dg.splitmix64(7, 4, rows))
    assert not np.array_equal(a, dg.splitmix64(8, 3, rows))


def _run_of(ends, rows):
    return np.searchsorted(ends.astype(np.int64), rows, side="right")


def test_nested_runs_are_nested_and_sorted():
    n = 2_000_000
    t, plan = dg.nested(n, seed=11)
    c1, c2, c3 = t.columns[:3]
    for c in (c1, c2, c3):
        assert int(c.run_ends[-1]) == n and np.all(np.diff(c.run_ends.astype(np.int64)) > 0)
    assert np.isin(c1.run_ends, c2.run_ends).all()
    assert np.isin(c2.run_ends, c3.run_ends).all()
    # c2 strictly increasing inside every c1 run, c3 inside every c2 run
    for child, parent, dom in ((c2, c1, 10_000), (c3, c2, 1_000)):
        par = _run_of(parent.run_ends, child.run_ends.astype(np.int64) - 1)
        same_parent = par[1:] == par[:-1]
        assert np.all(np.diff(child.run_values.astype(np.int64))[same_parent] > 0)
        assert child.run_values.min() >= 0 and child.run_values.max() < dom
    assert np.array_equal(c1.run_values, np.arange(c1.run_values.shape[0]))
    mean3 = n / c3.run_ends.shape[0]
    assert 80 < mean3 < 110


def test_nested_codes_follow_their_definition():
    n = 300_000
    t, _ = dg.nested(n, seed=4)
    e3 = t.columns[2].run_ends
    rows = np.arange(n)
    per_row = dg.nested_codes4(4, e3, rows)
    assert np.array_equal(dg.nested_codes4_all(4, e3, n), per_row)
    # unpack the stored 4-bit codes and compare
    w = t.columns[3].words.astype(np.uint64)
    bit = rows.astype(np.uint64) * np.uint64(4)
    stored = (w[(bit >> np.uint64(5)).astype(np.int64)] >> (bit & np.uint64(31))) & np.uint64(15)
    assert np.array_equal(stored.astype(np.uint32), per_row)
    # non-decreasing inside every c3 run, 0..15
    run = _run_of(e3, rows)
    same_run = run[1:] == run[:-1]
    assert np.all(np.diff(per_row.astype(np.int64))[same_run] >= 0)
    assert per_row.max() <= 15


def test_nested_measures_and_lean_layout():
    t, plan = dg.nested(10_000, seed=2)
    lt, lplan = dg.nested(10_000, seed=2, lean=True)
    assert [c.enc for c in t.columns] == ["rle", "rle", "rle", "dict", "dict", "dict", "packed", "packed"]
    assert [c.enc for c in lt.columns] == ["rle", "rle", "rle", "dict", "packed", "packed"]
    assert t.columns[6].base == dg.NESTED_BASE7 and t.columns[6].bit_width == 8
    assert t.columns[7].base == dg.NESTED_BASE8 and t.columns[7].bit_width == 12
    assert np.array_equal(t.columns[6].words, lt.columns[4].words)
    assert plan.aggs[0].col == 6 and lplan.aggs[0].col == 4
    assert plan.preds[0].col == 2 and plan.group_by == [1, 3]


def test_batch_queries_alternate_templates():
    rng = np.random.default_rng(0)
    qs = dg.batch_queries(rng, 100, 8)
    assert sum(k == "tiny" for _, k, _ in qs) == 50
    assert all(0 <= p < 8 for p, _, _ in qs)
    sizes = dg.partition_sizes(rng, 1000)
    assert sizes.min() >= 10_000 and sizes.max() <= 50_000_000


def test_subtable_is_the_selected_rows():
    n = 50_000
    full, _ = dg.nested(n, seed=6, lean=True)
    runs = full.columns[:3]
    ranges = [(0, 100), (1234, 5000), (49_990, 50_000)]
    sub = dg.nested_subtable(runs, 6, ranges)
    rows = np.concatenate([np.arange(a, b) for a, b in ranges])
    from oracle import oracle
    for j in range(6):
        np.testing.assert_array_equal(oracle.decode(sub.columns[j]), oracle.decode(full.columns[j])[rows])
    pre = dg.nested_subtable(runs, 6, [(0, n)])
    for j in range(6):
        np.testing.assert_array_equal(oracle.decode(pre.columns[j]), oracle.decode(full.columns[j]))
    c2 = runs[1]
    v = int(c2.run_values[c2.run_values.shape[0] // 2])
    vr = dg.value_ranges(c2, v)
    dec = oracle.decode(c2)
    assert sum(b - a for a, b in vr) == int((dec == v).sum())
    assert all((dec[a:b] == v).all() for a, b in vr)
