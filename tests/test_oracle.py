"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
worked example printed in the paper (tests/golden, each with its citation),
a closed form, an invariant, a library routine (numpy's repeat / unique /
ufunc.at, i.e. the paper's own tensor formulation in tests/tensor_ref.py),
Python's exact integers and correctly rounded int->float conversion, or brute
force over every tiny table.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests import tensor_ref
from tests.helpers import as_plain, mask_rle, random_column, random_plan, rle_inclusive

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def assert_same(o, ref):
    keys, aggs, overflow = ref
    assert (o.status == -6) == overflow
    assert len(o.keys) == len(keys)
    for a, b in zip(o.keys, keys):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(o.aggs, aggs):
        if a.dtype == np.float64:
            np.testing.assert_array_equal(a, np.asarray(b, dtype=np.float64))   # bit-exact AVG
        else:
            np.testing.assert_array_equal(a, np.asarray(b).astype(a.dtype))


# ---------------------------------------------------------------- paper examples
def test_primitive_examples_pin_the_tensor_reference():
    """Section 2.2 examples pin the numpy stand-ins of repeat_interleave,
    unique and scatter that tests/tensor_ref.py is built from."""
    g = load("primitives_examples.json")
    ri = g["repeat_interleave"]
    assert np.repeat(ri["input"], ri["repeats"]).tolist() == ri["result"]
    u, inv = np.unique(g["unique"]["input"], return_inverse=True)
    assert u.tolist() == g["unique"]["unique"] and inv.tolist() == g["unique"]["inverse"]
    sc = g["scatter_sum"]
    out = np.zeros(max(sc["index"]) + 1, dtype=np.int64)
    np.add.at(out, sc["index"], sc["src"])
    assert out.tolist() == sc["result"]


def test_alignment_example(oracle_mod):
    g = load("alignment_example.json")
    c1 = rle_inclusive(g["c1"]["val"], g["c1"]["start"], g["c1"]["end"])
    c2 = rle_inclusive(g["c2"]["val"], g["c2"]["start"], g["c2"]["end"])
    seg, ridx = oracle_mod.align([c1.run_ends, c2.run_ends], c1.n_rows)
    al = g["aligned"]
    assert (seg - 1).tolist() == al["end"]
    assert np.concatenate([[0], seg[:-1]]).tolist() == al["start"]
    r1 = c1.run_values[ridx[0]]
    r2 = c2.run_values[ridx[1]]
    assert r1.tolist() == al["r1_val"] and r2.tolist() == al["r2_val"]
    assert (r1 + r2).tolist() == al["sum"]
    # the same segments seen through a grouped query: one group per aligned
    # segment, COUNT = its length
    t = dg.Table([c1, c2], c1.n_rows)
    o = oracle_mod.query(t, dg.Plan([], [0, 1], [dg.Agg("count")]))
    lens = {(a, b): e - s + 1 for a, b, s, e in zip(al["r1_val"], al["r2_val"], al["start"], al["end"])}
    got = {(int(a), int(b)): int(c) for a, b, c in zip(o.keys[0], o.keys[1], o.aggs[0])}
    assert got == lens


def test_groupby_example(oracle_mod):
    g = load("groupby_example.json")
    a = rle_inclusive(g["A"]["val"], g["A"]["start"], g["A"]["end"])
    b = rle_inclusive(g["B"]["val"], g["B"]["start"], g["B"]["end"])
    t = dg.Table([a, b], a.n_rows)
    o = oracle_mod.query(t, dg.Plan([], [0], [dg.Agg("sum", 1)]))
    assert o.keys[0].tolist() == g["result"]["keys"]
    assert o.aggs[0].tolist() == g["result"]["sum"]
    seg, ridx = oracle_mod.align([a.run_ends, b.run_ends], a.n_rows)
    al = g["aligned"]
    lens = np.diff(np.concatenate([[0], seg]))
    assert lens.tolist() == al["len"]
    assert b.run_values[ridx[1]].tolist() == al["B_val"]
    assert (b.run_values[ridx[1]] * lens).tolist() == al["v_times_l"]


def test_encoding_examples(oracle_mod):
    g = load("encoding_examples.json")["plain_to_rle"]
    col = rle_inclusive(g["v"], g["s"], g["e"])
    assert oracle_mod.decode(col).tolist() == g["plain"]
    g = load("encoding_examples.json")["plain_to_plain_index"]
    idx = dg.Index(np.array(g["outlier_values"]), np.array(g["outlier_positions"]), 0, len(g["plain"]))
    got = oracle_mod.decode(idx)
    pos = np.array(g["outlier_positions"])
    assert got[pos].tolist() == g["outlier_values"]
    assert np.all(np.delete(got, pos) == 0)


def test_index_in_rle_example(oracle_mod):
    """Positions of an Index column that fall in RLE ranges [0-2], [6-7]:
    SUM over the index column under the range mask sees exactly p_out."""
    g = load("index_in_rle_example.json")
    n = g["n_rows"]
    m = mask_rle(list(zip(g["rle"]["start"], g["rle"]["end"])), n)
    pos = np.array(g["idx_pos"], dtype=np.int64)
    vals = (np.arange(pos.shape[0]) + 1) * 10 ** np.arange(pos.shape[0])   # 1, 20, 300: distinct digits
    x = dg.Index(vals.astype(np.int64), pos, 0, n)
    o = oracle_mod.query(dg.Table([m, x], n), dg.Plan([dg.Pred(0, "eq", 1)], [], [dg.Agg("sum", 1)]))
    expect = sum(int(v) for p, v in zip(pos, vals) if p in g["p_out"])
    assert int(o.aggs[0][0]) == expect


def test_range_intersect_example(oracle_mod):
    g = load("range_intersect_example.json")
    n = g["n_rows"]
    m1 = mask_rle(list(zip(g["c1"]["start"], g["c1"]["end"])), n)
    # c2's three ranges are adjacent, so as a data column they are three
    # separate runs of value 1 (non-maximal runs are allowed)
    v2 = [0] + [1, 1, 1]
    m2 = rle_inclusive(v2, [0] + g["c2"]["start"], [g["c2"]["start"][0] - 1] + g["c2"]["end"], n)
    seg, ridx = oracle_mod.align([m1.run_ends, m2.run_ends], n)
    starts = np.concatenate([[0], seg[:-1]])
    both = (m1.run_values[ridx[0]] == 1) & (m2.run_values[ridx[1]] == 1)
    assert starts[both].tolist() == g["result"]["s"]
    assert (seg[both] - 1).tolist() == g["result"]["e"]
    o = oracle_mod.query(dg.Table([m1, m2], n), dg.Plan([dg.Pred(0, "eq", 1), dg.Pred(1, "eq", 1)], [], [dg.Agg("count")]))
    assert int(o.aggs[0][0]) == sum(e - s + 1 for s, e in zip(g["result"]["s"], g["result"]["e"]))


def test_not_examples(oracle_mod):
    g = load("not_examples.json")
    r = g["not_rle"]
    n = r["total_size"]
    m = mask_rle(list(zip(r["s"], r["e"])), n)
    t = dg.Table([m, as_plain(np.arange(n))], n)
    o = oracle_mod.query(t, dg.Plan([dg.Pred(0, "ne", 1)], [], [dg.Agg("count"), dg.Agg("min", 1), dg.Agg("max", 1)]))
    assert int(o.aggs[0][0]) == sum(e - s + 1 for s, e in zip(r["result_s"], r["result_e"]))
    assert int(o.aggs[1][0]) == r["result_s"][0] and int(o.aggs[2][0]) == r["result_e"][-1]
    r = g["not_index"]
    n = r["total_size"]
    x = dg.Index(np.ones(len(r["p"]), dtype=np.int64), np.array(r["p"]), 0, n)
    t = dg.Table([x, as_plain(np.arange(n))], n)
    o = oracle_mod.query(t, dg.Plan([dg.Pred(0, "eq", 0)], [], [dg.Agg("count"), dg.Agg("sum", 1)]))
    rows = [i for s, e in zip(r["result_s"], r["result_e"]) for i in range(s, e + 1)]
    assert int(o.aggs[0][0]) == len(rows) and int(o.aggs[1][0]) == sum(rows)


# ---------------------------------------------------------------- decoders
@pytest.mark.parametrize("w", [1, 2, 3, 5, 7, 8, 13, 14, 16, 20, 31, 32, 33, 40, 47, 63, 64])
def test_bitpacked_decode_against_bigint_stream(oracle_mod, w):
    rng = np.random.default_rng(w)
    n = 97
    mask = (1 << w) - 1
    vals = [int(x) & mask for x in rng.integers(0, 2**63, size=n, dtype=np.uint64)]
    vals[0] = mask
    stream = 0
    for i, v in enumerate(vals):
        stream |= v << (i * w)
    nw = (n * w + 31) // 32 + 1
    words = np.array([(stream >> (32 * k)) & 0xFFFFFFFF for k in range(nw)], dtype=np.uint32)
    base = -12345
    col = dg.Packed(words, w, base, n)
    got = oracle_mod.decode(col)
    want = np.array([(v + base) - (1 << 64) if v + base >= 2**63 else v + base for v in vals], dtype=np.int64)
    np.testing.assert_array_equal(got, want)
    # a window in the middle
    np.testing.assert_array_equal(oracle_mod.decode(col, 10, 60), want[10:60])


def test_rle_decode_is_repeat(oracle_mod):
    rng = np.random.default_rng(3)
    for mean in (1.0, 2.5, 40.0):
        ends = dg.geometric_ends(rng, 5000, mean, np.int64)
        vals = rng.integers(-9, 9, size=ends.shape[0])
        col = dg.RLE(vals, ends, 5000)
        lens = np.diff(np.concatenate([[0], ends]))
        assert lens.sum() == 5000 and np.all(lens >= 1)               # run lengths sum to N
        np.testing.assert_array_equal(oracle_mod.decode(col), np.repeat(vals, lens))
        np.testing.assert_array_equal(oracle_mod.decode(col, 1234, 4321), np.repeat(vals, lens)[1234:4321])


# ---------------------------------------------------------------- against the paper's tensor formulation
ENCS = ["rle", "plain", "packed", "index", "dict"]


@pytest.mark.parametrize("seed", range(40))
def test_random_tables_match_tensor_formulation(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 300))
    ncol = int(rng.integers(1, 5))
    cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(ncol)]
    t = dg.Table(cols, n)
    plan = random_plan(rng, t)
    o = oracle_mod.query(t, plan)
    assert_same(o, tensor_ref.query(t, plan))
    # chunking over threads and row ranges changes nothing
    o2 = oracle_mod.query(t, plan, n_threads=3, row_ranges=[(0, n // 3), (n // 3, n)])
    assert_same(o2, tensor_ref.query(t, plan))


def test_large_chunked_scan_matches_tensor_formulation(oracle_mod):
    """Spans several 1M-row chunks of the oracle's scan."""
    rng = np.random.default_rng(77)
    n = 2_500_000
    a = dg.make_rle(rng, n, 50.0, 0, 9, np.int64, np.int64)
    b = dg.Plain(rng.integers(0, 100, size=n).astype(np.int64))
    t = dg.Table([a, b], n)
    plan = dg.Plan([dg.Pred(1, "lt", 30)], [0], [dg.Agg("sum", 1), dg.Agg("count"), dg.Agg("max", 1)])
    o = oracle_mod.query(t, plan, n_threads=4)
    av = np.repeat(a.run_values, np.diff(np.concatenate([[0], a.run_ends])))
    m = b.values < 30
    u, inv = np.unique(av[m], return_inverse=True)
    s = np.zeros(u.shape[0], dtype=np.int64)
    np.add.at(s, inv, b.values[m])
    mx = np.full(u.shape[0], -1, dtype=np.int64)
    np.maximum.at(mx, inv, b.values[m])
    np.testing.assert_array_equal(o.keys[0], u)
    np.testing.assert_array_equal(o.aggs[0], s)
    np.testing.assert_array_equal(o.aggs[1], np.bincount(inv).astype(np.uint64))
    np.testing.assert_array_equal(o.aggs[2], mx)


# ---------------------------------------------------------------- closed forms and invariants
def test_sum_over_rle_is_dot_of_values_and_lengths(oracle_mod):
    rng = np.random.default_rng(5)
    n = 100_000
    a = dg.make_rle(rng, n, 13.0, -1000, 1000, np.int64, np.int64)
    lens = np.diff(np.concatenate([[0], a.run_ends]))
    o = oracle_mod.query(dg.Table([a], n), dg.Plan([], [], [dg.Agg("sum", 0), dg.Agg("count")]))
    assert int(o.aggs[0][0]) == int(np.dot(a.run_values, lens))
    assert int(o.aggs[1][0]) == n


def test_single_run_column(oracle_mod):
    n = 12345
    a = dg.RLE(np.array([-7], dtype=np.int64), np.array([n], dtype=np.int64), n)
    o = oracle_mod.query(dg.Table([a], n), dg.Plan([], [0], [dg.Agg("sum", 0), dg.Agg("min", 0), dg.Agg("avg", 0)]))
    assert o.keys[0].tolist() == [-7]
    assert int(o.aggs[0][0]) == -7 * n and int(o.aggs[1][0]) == -7 and o.aggs[2][0] == -7.0


def test_invariants_on_the_tiny_workload(oracle_mod):
    t, plan = dg.tiny_two_rle(200_000, seed=11)
    plan = dg.Plan(plan.preds, plan.group_by, plan.aggs + [dg.Agg("min", 0), dg.Agg("max", 0), dg.Agg("avg", 0)])
    o = oracle_mod.query(t, plan)
    a, b = t.columns
    seg, ridx = oracle_mod.align([a.run_ends, b.run_ends], t.n_rows)
    lens = np.diff(np.concatenate([[0], seg]))
    assert np.all(lens > 0) and lens.sum() == t.n_rows                 # segments partition [0, N)
    boundaries = set(a.run_ends.tolist()) | set(b.run_ends.tolist())
    assert set(seg.tolist()) == boundaries                             # exactly the common refinement
    av = a.run_values[ridx[0]]
    passing = av < 50
    assert int(o.aggs[1].sum()) == int(lens[passing].sum())            # sum of COUNT = passing rows
    assert int(o.aggs[0].sum()) == int((av[passing].astype(np.int64) * lens[passing]).sum())
    assert np.all(o.aggs[2] <= o.aggs[4]) and np.all(o.aggs[4] <= o.aggs[3])   # MIN <= AVG <= MAX
    assert np.all(o.keys[0][1:] > o.keys[0][:-1])                      # ascending keys


# ---------------------------------------------------------------- metamorphic re-encodings
def test_reencoding_leaves_results_unchanged(oracle_mod):
    rng = np.random.default_rng(9)
    n = 3000
    vals = np.repeat(rng.integers(0, 40, size=300), rng.integers(1, 20, size=300))[:n]
    n = vals.shape[0]
    other = rng.integers(-5, 5, size=n).astype(np.int64)
    v, e = dg.rle_encode(vals, np.int64)
    encs = {
        "rle": dg.RLE(v.astype(np.int64), e, n),
        "plain": dg.Plain(vals.astype(np.int64)),
        "packed": dg.make_packed((vals - 0).astype(np.uint64), 6, 0),
        "index": dg.Index(vals[vals != 7].astype(np.int64), np.flatnonzero(vals != 7).astype(np.int64), 7, n),
    }
    # non-maximal runs: split every run in two where possible
    split_ends = np.unique(np.concatenate([e, np.maximum(1, e - 1)]))
    encs["rle_split"] = dg.RLE(vals[split_ends - 1].astype(np.int64), split_ends.astype(np.int64), n)
    plan = dg.Plan([dg.Pred(0, "between", 5, 30), dg.Pred(1, "ne", 0)], [0],
                   [dg.Agg("sum", 1), dg.Agg("count"), dg.Agg("min", 0), dg.Agg("max", 0), dg.Agg("avg", 0)])
    results = []
    for name, col in encs.items():
        o = oracle_mod.query(dg.Table([col, dg.Plain(other)], n), plan)
        results.append((name, o))
    base = results[0][1]
    for name, o in results[1:]:
        for x, y in zip(base.keys + base.aggs, o.keys + o.aggs):
            np.testing.assert_array_equal(x, y, err_msg=name)
    # permuting column order changes nothing
    o = oracle_mod.query(dg.Table([dg.Plain(other), encs["rle"]], n),
                         dg.Plan([dg.Pred(1, "between", 5, 30), dg.Pred(0, "ne", 0)], [1],
                                 [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 1), dg.Agg("max", 1), dg.Agg("avg", 1)]))
    for x, y in zip(base.keys + base.aggs, o.keys + o.aggs):
        np.testing.assert_array_equal(x, y)


def test_row_shards_merge_to_the_whole(oracle_mod):
    """Splitting the rows into shards and merging partial groups gives the
    whole result (the exact merge a row-range shard would need)."""
    t, plan = dg.tiny_two_rle(50_000, seed=4)
    whole = oracle_mod.query(t, plan)
    parts = [oracle_mod.query(t, plan, row_ranges=[(s, min(s + 7001, t.n_rows))]) for s in range(0, t.n_rows, 7001)]
    acc = {}
    for p in parts:
        for k, s, c in zip(p.keys[0], p.aggs[0], p.aggs[1]):
            a = acc.setdefault(int(k), [0, 0])
            a[0] += int(s)
            a[1] += int(c)
    assert sorted(acc) == whole.keys[0].tolist()
    assert [acc[k][0] for k in sorted(acc)] == whole.aggs[0].tolist()
    assert [acc[k][1] for k in sorted(acc)] == whole.aggs[1].tolist()


# ---------------------------------------------------------------- exactness
def test_sum_overflow_is_reported_and_avg_is_exact(oracle_mod):
    big = 2**62 + 12345
    a = dg.RLE(np.array([big, -3], dtype=np.int64), np.array([3, 4], dtype=np.int64), 4)
    o = oracle_mod.query(dg.Table([a], 4), dg.Plan([], [], [dg.Agg("sum", 0)]))
    assert o.status == -6
    lo, hi = o.sum128[0]
    exact = 3 * big - 3
    assert (int(hi[0]) << 64) + int(lo[0]) == exact
    o = oracle_mod.query(dg.Table([a], 4), dg.Plan([], [], [dg.Agg("avg", 0)]))
    assert o.status == 0 and o.aggs[0][0] == float(exact) / 4.0


@pytest.mark.parametrize("total,count", [(2**53 + 1, 1), (2**60 + 3, 3), (-(2**64) - 1, 7), (10**20 + 1, 3), (12345, 0)])
def test_avg_rounds_the_exact_sum_once(oracle_mod, total, count):
    """AVG = double(exact SUM) / double(COUNT), with the 128-bit sum rounded
    to nearest even, as Python's int -> float conversion does."""
    if count == 0:
        a = dg.Plain(np.array([5], dtype=np.int64))
        o = oracle_mod.query(dg.Table([a], 1), dg.Plan([dg.Pred(0, "lt", 0)], [], [dg.Agg("avg", 0), dg.Agg("count")]))
        assert o.aggs[0][0] == 0.0 and int(o.aggs[1][0]) == 0
        return
    q, r = divmod(total, count)
    parts = [q] * count
    parts[0] += r
    while any(not (-2**63 <= p < 2**63) for p in parts):
        parts = [p // 2 for p in parts] + [p - p // 2 for p in parts]
    a = dg.Plain(np.array(parts, dtype=np.int64))
    o = oracle_mod.query(dg.Table([a], len(parts)), dg.Plan([], [], [dg.Agg("avg", 0)]))
    assert o.aggs[0][0] == float(total) / float(len(parts))


# ---------------------------------------------------------------- brute force
def test_brute_force_every_tiny_table(oracle_mod):
    """Every table of N <= 4 rows with A in {0,1,2}^N (RLE, maximal runs) and
    B in {0,1}^N (plain): SELECT B, SUM(A), COUNT(*), MIN(A) WHERE A >= 1 GROUP BY B."""
    plan = dg.Plan([dg.Pred(0, "ge", 1)], [1], [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 0)])
    for n in range(1, 5):
        for av in itertools.product([0, 1, 2], repeat=n):
            v, e = dg.rle_encode(np.array(av, dtype=np.int64), np.int64)
            for bv in itertools.product([0, 1], repeat=n):
                t = dg.Table([dg.RLE(v, e, n), dg.Plain(np.array(bv, dtype=np.int64))], n)
                o = oracle_mod.query(t, plan)
                groups = {}
                for x, y in zip(av, bv):
                    if x >= 1:
                        g = groups.setdefault(y, [0, 0, 99])
                        g[0] += x
                        g[1] += 1
                        g[2] = min(g[2], x)
                assert o.keys[0].tolist() == sorted(groups)
                assert o.aggs[0].tolist() == [groups[k][0] for k in sorted(groups)]
                assert o.aggs[1].tolist() == [groups[k][1] for k in sorted(groups)]
                assert o.aggs[2].tolist() == [groups[k][2] for k in sorted(groups)]


# ---------------------------------------------------------------- strings and validation
def test_dictionary_predicates_compare_bytes(oracle_mod):
    strings = sorted([b"a", b"ab", b"abc", b"b", b"ba", b"zz", b"\xff"])
    rng = np.random.default_rng(2)
    codes = rng.integers(0, len(strings), size=500).astype(np.uint64)
    d = dg.make_dict(strings, codes, 3)
    t = dg.Table([d], 500)
    cases = [("lt", [b"ab"]), ("le", [b"ab"]), ("gt", [b"b"]), ("ge", [b"aa"]), ("eq", [b"ba"]),
             ("ne", [b"ba"]), ("between", [b"ab", b"b"]), ("in", [b"zz", b"q", b"a"])]
    for op, lits in cases:
        o = oracle_mod.query(t, dg.Plan([dg.Pred(0, op, strs=lits)], [0], [dg.Agg("count"), dg.Agg("min", 0), dg.Agg("max", 0)]))
        s = [strings[c] for c in codes]
        f = {"lt": lambda x: x < lits[0], "le": lambda x: x <= lits[0], "gt": lambda x: x > lits[0],
             "ge": lambda x: x >= lits[0], "eq": lambda x: x == lits[0], "ne": lambda x: x != lits[0],
             "between": lambda x: lits[0] <= x <= lits[1], "in": lambda x: x in lits}[op]
        keep = sorted(set(x for x in s if f(x)))
        assert [strings[k] for k in o.keys[0]] == keep, op
        assert o.aggs[0].tolist() == [sum(1 for x in s if x == k) for k in keep]


@pytest.mark.parametrize("bad", ["unsorted_ends", "short_ends", "pos_out_of_range", "pos_unsorted", "few_words", "code_range"])
def test_malformed_columns_are_rejected(oracle_mod, bad):
    n = 10
    cols = {
        "unsorted_ends": dg.RLE(np.array([1, 2]), np.array([6, 4]), n),
        "short_ends": dg.RLE(np.array([1, 2]), np.array([4, 9]), n),
        "pos_out_of_range": dg.Index(np.array([1]), np.array([10]), 0, n),
        "pos_unsorted": dg.Index(np.array([1, 2]), np.array([5, 3]), 0, n),
        "few_words": dg.Packed(np.zeros(2, dtype=np.uint32), 7, 0, n),
        "code_range": dg.make_dict([b"x", b"y", b"z"], np.full(n, 3, dtype=np.uint64), 2),
    }
    with pytest.raises(ValueError):
        oracle_mod.query(dg.Table([cols[bad]], n), dg.Plan([], [], [dg.Agg("sum" if bad != "code_range" else "min", 0)]))
