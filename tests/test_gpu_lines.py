"""GPU parity for the run-line group table: GROUP BY an RLE column first (its
runs long next to a tile) and row-level columns after it.  The specialised
row kernel then gives each run a line of the shared table and recovers the
run's key at the flush.  Covered here: tiles with more runs than lines (they
fall back to the global accumulators), flushes forced by line reuse, by the
flush period and at launch splits, an IN list on the run key (remapped
digits), three keys, sorted inner keys (warp pre-reduction), and tables whose
runs are too short for lines.  The bar is bit-exact equality with the CPU
oracle."""
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


@pytest.fixture(scope="module")
def ctx(cq):
    return cq.cq_ctx_create(0)


def run(cq, ctx, table, plan, opts=None):
    t, cols = cq.table_from(ctx, table)
    return cq.fetch_all(cq.cq_query_run(t, plan, opts=opts))


def check(got, ref, msg=""):
    want = ref.keys + ref.aggs
    assert len(got) == len(want), msg
    for i, (g, w) in enumerate(zip(got, want)):
        assert g.dtype == w.dtype, (msg, i, g.dtype, w.dtype)
        np.testing.assert_array_equal(g, w, err_msg=f"{msg} output column {i}")


def rle_with_short_stretch(rng, n, mean, lo, hi, short_from, short_to):
    """Runs of mean length `mean`, except unit runs over [short_from, short_to)."""
    ends = dg.geometric_ends(rng, n, mean, np.int64)
    ends = ends[(ends <= short_from) | (ends >= short_to)]
    ends = np.unique(np.concatenate([ends, np.arange(short_from + 1, short_to + 1, dtype=np.int64), [n]]))
    vals = rng.integers(lo, hi + 1, size=ends.shape[0]).astype(np.int64)
    return dg.RLE(vals, ends, n)


AGGS = [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("min", 2), dg.Agg("max", 3), dg.Agg("avg", 3)]


@pytest.mark.parametrize("mean", [300.0, 1000.0, 20000.0])
def test_run_key_then_plain_key(cq, ctx, oracle_mod, mean):
    rng = np.random.default_rng(int(mean))
    n = 1_500_007
    a = dg.make_rle(rng, n, mean, 0, 999, np.int32, np.int32)
    b = dg.Plain(rng.integers(0, 50, size=n).astype(np.int32))
    v = dg.Plain(rng.integers(-1000, 1000, size=n).astype(np.int64))
    w = dg.make_packed(rng.integers(0, 1 << 20, size=n).astype(np.uint64), 20, 1 << 33)
    table = dg.Table([a, b, v, w], n)
    for preds in ([], [dg.Pred(2, "lt", 500)], [dg.Pred(0, "between", 100, 800), dg.Pred(2, "gt", -900)]):
        plan = dg.Plan(preds, [0, 1], AGGS)
        ref = oracle_mod.query(table, plan, n_threads=4)
        check(run(cq, ctx, table, plan), ref, f"mean {mean} {preds}")


def test_tiles_with_more_runs_than_lines(cq, ctx, oracle_mod):
    """A stretch of unit runs: its tiles hold thousands of runs and take the
    global-accumulator fallback; the tiles around it use lines."""
    rng = np.random.default_rng(5)
    n = 2_000_003
    a = rle_with_short_stretch(rng, n, 2000.0, 0, 499, 700_000, 760_000)
    b = dg.Plain(rng.integers(0, 30, size=n).astype(np.int32))
    v = dg.Plain(rng.integers(-50, 50, size=n).astype(np.int64))
    w = dg.Plain(rng.integers(0, 10_000, size=n).astype(np.int32))
    table = dg.Table([a, b, v, w], n)
    plan = dg.Plan([dg.Pred(3, "lt", 7000)], [0, 1], AGGS)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "short stretch")


def test_in_list_on_the_run_key_and_three_keys(cq, ctx, oracle_mod):
    """Key 0's digits come from an IN list's ranks (remapped at the flush);
    lines two keys wide."""
    rng = np.random.default_rng(9)
    n = 1_200_001
    a = dg.make_rle(rng, n, 800.0, 0, 5000, np.int64, np.int64)
    strings = sorted({bytes(rng.choice(list(b"abcdefgh"), size=int(rng.integers(2, 6)))) for _ in range(200)})
    codes = rng.integers(0, len(strings), size=n).astype(np.uint64)
    d = dg.make_dict(strings, codes, 8)
    c = dg.make_packed(rng.integers(0, 6, size=n).astype(np.uint64), 3, -2)
    v = dg.Plain(rng.integers(-(1 << 40), 1 << 40, size=n).astype(np.int64))
    table = dg.Table([a, d, c, v], n)
    ins = [int(x) for x in rng.choice(5001, size=300, replace=False)]
    aggs = [dg.Agg("count"), dg.Agg("sum", 3), dg.Agg("min", 3), dg.Agg("max", 1)]
    for gb in ([0, 2], [0, 1, 2], [0, 2, 1]):
        plan = dg.Plan([dg.Pred(0, "in", ints=ins)], gb, aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"in, keys {gb}")
    plan = dg.Plan([dg.Pred(1, "lt", strs=[b"d"])], [0, 2], [dg.Agg("count"), dg.Agg("avg", 3)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "2 keys")


def test_sorted_inner_key_prereduction(cq, ctx, oracle_mod):
    """Nested-style data: the inner key is non-decreasing inside each run of
    the run key, so runs of equal groups are reduced across the warp first."""
    table, plan = dg.nested(3_000_000, seed=44, lean=True)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "nested")


@pytest.mark.parametrize("rows", [65536, 300_000])
def test_lines_across_split_launches(cq, ctx, oracle_mod, rows):
    old = os.environ.get("CQ_LAUNCH_ROWS")
    os.environ["CQ_LAUNCH_ROWS"] = str(rows)
    try:
        table, plan = dg.heterogeneous(1_000_003, seed=23)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"split {rows}")
    finally:
        if old is None:
            del os.environ["CQ_LAUNCH_ROWS"]
        else:
            os.environ["CQ_LAUNCH_ROWS"] = old


def test_short_runs_keep_the_hash_table(cq, ctx, oracle_mod):
    rng = np.random.default_rng(12)
    n = 500_001
    a = dg.make_rle(rng, n, 3.0, 0, 3000, np.int32, np.int32)
    b = dg.Plain(rng.integers(0, 40, size=n).astype(np.int32))
    v = dg.Plain(rng.integers(-9, 9, size=n).astype(np.int64))
    table = dg.Table([a, b, v, v], n)
    plan = dg.Plan([], [0, 1], AGGS)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "short runs")


@pytest.mark.parametrize("seed", range(4))
def test_in_place_groups_with_holes(cq, ctx, oracle_mod, seed):
    """Sorted keys and a filter that passes rows in stretches: most 32-row
    groups pass whole and are aggregated in place; the stretches' edges leave
    groups with holes, where a run of equal keys must not span a failing row."""
    rng = np.random.default_rng(300 + seed)
    n = 700_001
    key = dg.Plain((np.arange(n) // int(rng.integers(3, 40))).astype(np.int32) % 4000)
    sel = dg.make_rle(rng, n, float(rng.choice([20.0, 70.0, 300.0])), 0, 9, np.int32, np.int32)
    v = dg.make_packed(rng.integers(0, 1 << 10, size=n).astype(np.uint64), 10, 5)
    w = dg.Plain(rng.integers(-500, 500, size=n).astype(np.int32))
    table = dg.Table([key, sel, v, w], n)
    aggs = [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("sum", 3), dg.Agg("min", 3), dg.Agg("max", 2)]
    for preds in ([dg.Pred(1, "lt", 6)], [dg.Pred(1, "ne", 3), dg.Pred(3, "gt", -450)]):
        plan = dg.Plan(preds, [0], aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"seed {seed} {preds}")
        plan = dg.Plan(preds, [1, 0], aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"seed {seed} {preds} rle key")
        # SUMs of non-negative inputs only: the packed prefix sums
        plan = dg.Plan(preds, [0], [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("avg", 2)])
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"seed {seed} {preds} packed")
