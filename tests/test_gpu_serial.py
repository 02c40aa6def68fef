"""GPU parity for the serial walk of sorted data (Section 7: an aggregate over
a stretch of equal groups is one update).  The specialised row kernel takes
it when the filter is decided by pass bitmaps of RLE / index columns alone,
every key but the run-line key and every aggregated value is a staged field
of at most 32 bits, and every aggregate reduces in 32 bits: each lane walks
8, 16 or 32 consecutive rows from registers.  Covered: run-line keys (lines
advancing inside a lane's rows; tiles with more runs than lines taking the
row path), dense and hashed shared tables, 4-, 8-, 12-, 13-, 14-bit and
plain 32-bit fields, negative values, MIN / MAX, OR and NOT over pass
bitmaps, index-column filters and ragged tails.  The bar is bit-exact
equality with the CPU oracle."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.test_gpu_lines import rle_with_short_stretch

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


@pytest.mark.parametrize("lo3, hi3", [(200, 699), (0, 999), (500, 510), (999, 0)])
def test_nested_query(cq, ctx, oracle_mod, lo3, hi3):
    """The nested table (c2 runs of ~1e4 rows, c4 non-decreasing inside c3
    runs): GROUP BY c2, c4 with SUMs of the 8- and 12-bit fields, COUNT,
    MIN and MAX, under stretches of passing c3 runs (none for lo3 > hi3)."""
    table, plan = dg.nested(1_000_003, seed=71, lo3=lo3, hi3=hi3, lean=True)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "nested")
    p = dg.Plan(plan.preds, plan.group_by, plan.aggs + [dg.Agg("count"), dg.Agg("min", 5), dg.Agg("max", 4),
                                                        dg.Agg("avg", 5)])
    check(run(cq, ctx, table, p), oracle_mod.query(table, p, n_threads=4), "nested, more aggregates")


@pytest.mark.parametrize("card", [37, 4000, 300_000])
@pytest.mark.parametrize("widths", [(4, 8, 12), (14, 8, 12), (13, 3, 32)])
def test_sorted_key_and_field_widths(cq, ctx, oracle_mod, card, widths):
    """A sorted staged key (dense table for few groups, the shared hash
    table for many), values of several widths (lanes of 8, 16 or 32 rows),
    a plain int32 column with negative values, filters on an RLE column."""
    rng = np.random.default_rng(card * 7 + widths[0])
    n = 700_001
    kb, vb, wb = widths
    step = int(rng.integers(2, 30))
    keys = (np.arange(n, dtype=np.int64) // step) % min(card, 1 << kb)
    k = dg.make_dict([b"k%06d" % i for i in range(1 << kb)], np.sort(keys).astype(np.uint64), kb)
    sel = dg.make_rle(rng, n, 40.0, 0, 9, np.int32, np.int32)
    v = dg.make_packed(rng.integers(0, 1 << vb, size=n).astype(np.uint64), vb, 3)
    if wb == 32:
        w = dg.Plain(rng.integers(-(1 << 20), 1 << 20, size=n).astype(np.int32))
    else:
        w = dg.make_packed(rng.integers(0, 1 << wb, size=n).astype(np.uint64), wb, -7)
    table = dg.Table([k, sel, v, w], n)
    aggs = [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("sum", 3), dg.Agg("min", 3), dg.Agg("max", 2),
            dg.Agg("max", 3)]
    for preds in ([], [dg.Pred(1, "lt", 6)], [dg.Pred(1, "between", 3, 3)]):
        plan = dg.Plan(preds, [0], aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"{preds}")
    # plain int32 key (a 32-bit field)
    kp = dg.Plain(np.sort(rng.integers(-1000, 1000, size=n)).astype(np.int32))
    table = dg.Table([kp, sel, v, w], n)
    plan = dg.Plan([dg.Pred(1, "ne", 4)], [0], aggs)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "plain key")


def test_or_not_and_index_filters(cq, ctx, oracle_mod):
    """Filters of several pass bitmaps: OR groups, NOT, an index column
    (listed rows differ from the default), a program."""
    rng = np.random.default_rng(5)
    n = 900_007
    a = dg.make_rle(rng, n, 25.0, 0, 99, np.int32, np.int32)
    b = dg.make_rle(rng, n, 300.0, -50, 50, np.int64, np.int64)
    x = dg.make_index(rng, n, n // 20, 1, 9, default=0)
    key = dg.make_packed(np.sort(rng.integers(0, 200, size=n)).astype(np.uint64), 8, 0)
    v = dg.make_packed(rng.integers(0, 1 << 12, size=n).astype(np.uint64), 12, 1 << 33)
    table = dg.Table([a, b, x, key, v], n)
    aggs = [dg.Agg("count"), dg.Agg("sum", 4), dg.Agg("min", 4), dg.Agg("avg", 4)]
    cases = [
        ([dg.Pred(0, "lt", 30, group=1), dg.Pred(1, "gt", 40, group=1)], None),
        ([dg.Pred(0, "between", 10, 60, neg=True), dg.Pred(1, "lt", 0)], None),
        ([dg.Pred(2, "gt", 0)], None),
        ([dg.Pred(2, "eq", 0), dg.Pred(0, "ne", 7)], None),
        ([dg.Pred(0, "lt", 50), dg.Pred(1, "gt", 0), dg.Pred(2, "gt", 4)],
         [("pred", 0), ("pred", 1), ("and", 2), ("pred", 2), ("or", 2), ("not", 0)]),
    ]
    for preds, prog in cases:
        plan = dg.Plan(preds, [3], aggs, filter=prog)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"{preds} {prog}")


@pytest.mark.parametrize("mean", [150.0, 900.0])
def test_run_line_key_with_inner_key(cq, ctx, oracle_mod, mean):
    """GROUP BY an RLE column (run lines; with short runs the lines advance
    inside lanes' rows, and a stretch of unit runs gives tiles more runs than
    lines) and a sorted inner key; filter on a third RLE column."""
    rng = np.random.default_rng(int(mean))
    n = 1_500_001
    a = rle_with_short_stretch(rng, n, mean, 0, 3000, 600_000, 640_000)
    # inner key non-decreasing inside every run of a
    ends = a.run_ends.astype(np.int64)
    starts = np.concatenate([[0], ends[:-1]])
    off = np.arange(n, dtype=np.int64) - np.repeat(starts, ends - starts)
    inner = dg.make_packed((off // 7 % 16).astype(np.uint64), 4, 0)
    sel = dg.make_rle(rng, n, 200.0, 0, 3, np.int32, np.int32)
    v = dg.make_packed(rng.integers(0, 256, size=n).astype(np.uint64), 8, 100)
    w = dg.make_packed(rng.integers(0, 4096, size=n).astype(np.uint64), 12, -2048)
    table = dg.Table([a, inner, sel, v, w], n)
    aggs = [dg.Agg("sum", 3), dg.Agg("sum", 4), dg.Agg("count"), dg.Agg("max", 4), dg.Agg("min", 3)]
    for preds in ([dg.Pred(2, "lt", 3)], []):
        plan = dg.Plan(preds, [0, 1], aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"mean {mean} {preds}")


@pytest.mark.parametrize("n", [1, 31, 257, 8191, 8193, 65_537])
def test_ragged_and_tiny_tables(cq, ctx, oracle_mod, n):
    rng = np.random.default_rng(n)
    key = dg.make_packed(np.sort(rng.integers(0, 5, size=n)).astype(np.uint64), 4, 0)
    sel = dg.make_rle(rng, n, 9.0, 0, 1, np.int32, np.int32)
    v = dg.make_packed(rng.integers(0, 1 << 12, size=n).astype(np.uint64), 12, 0)
    table = dg.Table([key, sel, v], n)
    plan = dg.Plan([dg.Pred(1, "eq", 1)], [0], [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("max", 2)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), f"n {n}")
