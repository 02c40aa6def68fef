"""GPU parity for filters with OR and NOT (Section 5 logical operators on
masks; Appendix A.1 NOT): random filter programs and OR-group plans over
tables of every encoding, in every execution path (the specialised and the
generic row kernel, segment mode walking tiles and walking runs, expand then
scan, batches, the serving loop).  The bar is bit-exact equality with the
CPU oracle, which evaluates the program directly, row by row."""
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, random_or_groups, random_plan, random_tree

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ENCS = ["rle", "plain", "packed", "index", "dict"]


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


def with_filter(rng, plan, tree):
    """The plan with a random program (tree) or random OR groups."""
    if tree:
        return dg.Plan(plan.preds, plan.group_by, plan.aggs, filter=random_tree(rng, len(plan.preds)))
    return dg.Plan(random_or_groups(rng, plan.preds), plan.group_by, plan.aggs)


def test_not_examples(cq, ctx, oracle_mod):
    """Appendix A.1's NOT of an RLE and of an Index mask, on the device."""
    g = json.load(open(os.path.join(GOLDEN, "not_examples.json")))
    r = g["not_rle"]
    n = r["total_size"]
    from tests.helpers import mask_rle
    m = mask_rle(list(zip(r["s"], r["e"])), n)
    rows = dg.Plain(np.arange(n, dtype=np.int64))
    plan = dg.Plan([dg.Pred(0, "eq", 1, neg=True)], [1], [dg.Agg("count")])
    got = run(cq, ctx, dg.Table([m, rows], n), plan)
    assert got[0].tolist() == [i for s, e in zip(r["result_s"], r["result_e"]) for i in range(s, e + 1)]
    r = g["not_index"]
    x = dg.Index(np.ones(len(r["p"]), dtype=np.int64), np.array(r["p"], dtype=np.int64), 0, n)
    plan = dg.Plan([dg.Pred(0, "eq", 1)], [1], [dg.Agg("count")], filter=[("pred", 0), ("not", 0)])
    got = run(cq, ctx, dg.Table([x, rows], n), plan)
    assert got[0].tolist() == [i for s, e in zip(r["result_s"], r["result_e"]) for i in range(s, e + 1)]


@pytest.mark.parametrize("seed", range(48))
def test_random_filters(cq, ctx, oracle_mod, seed):
    """Random tables of every encoding (several tiles and a ragged tail),
    random predicates combined by a random program (even seeds) or random
    OR groups and negations (odd seeds); the specialised and the generic
    row kernel."""
    rng = np.random.default_rng(11000 + seed)
    n = int(rng.choice([1, 1000, 4097, 20000, 70001]))
    cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(int(rng.integers(2, 5)))]
    table = dg.Table(cols, n)
    plan = with_filter(rng, random_plan(rng, table, n_preds=int(rng.integers(1, 6))), seed % 2 == 0)
    ref = oracle_mod.query(table, plan)
    for kernel in (0, 1):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


@pytest.mark.parametrize("seed", range(24))
def test_random_filters_segment_mode(cq, ctx, oracle_mod, seed):
    """Every column RLE or index-encoded: segment mode, walking tiles (2)
    and walking runs (3)."""
    rng = np.random.default_rng(12000 + seed)
    n = int(rng.choice([5000, 40001, 200000]))
    cols = [random_column(rng, n, str(rng.choice(["rle", "index"]))) for _ in range(int(rng.integers(2, 4)))]
    table = dg.Table(cols, n)
    plan = with_filter(rng, random_plan(rng, table, n_preds=int(rng.integers(1, 5))), seed % 2 == 0)
    ref = oracle_mod.query(table, plan)
    for kernel in (2, 3):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


@pytest.mark.parametrize("seed", range(8))
def test_random_filters_expand_then_scan(cq, ctx, oracle_mod, seed):
    rng = np.random.default_rng(13000 + seed)
    n = int(rng.choice([3000, 50001]))
    cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(3)]
    table = dg.Table(cols, n)
    plan = with_filter(rng, random_plan(rng, table, n_preds=3), seed % 2 == 0)
    check(run(cq, ctx, table, plan, cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN)),
          oracle_mod.query(table, plan), f"dts seed {seed}")


def test_keys_under_or_and_not_are_not_narrowed(cq, ctx, oracle_mod):
    """A range or IN predicate on a group-by column narrows the key domain
    only when every passing row satisfies it: under OR or NOT rows outside
    it pass, and their keys must still be counted."""
    rng = np.random.default_rng(77)
    n = 60_001
    k = dg.Plain(rng.integers(0, 5000, size=n).astype(np.int64))
    r = dg.make_rle(rng, n, 6.0, 0, 4000, np.int64, np.int64)
    v = dg.Plain(rng.integers(-100, 100, size=n).astype(np.int64))
    table = dg.Table([k, r, v], n)
    aggs = [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("min", 2)]
    cases = [
        ([dg.Pred(0, "between", 100, 200, group=1), dg.Pred(2, "lt", -90, group=1)], None),
        ([dg.Pred(0, "between", 100, 4800, neg=True)], None),
        ([dg.Pred(0, "in", ints=[5, 77, 901]), dg.Pred(2, "gt", 95)], [("pred", 0), ("pred", 1), ("or", 2)]),
        ([dg.Pred(0, "in", ints=[5, 77, 901])], [("pred", 0), ("not", 0)]),
        ([dg.Pred(1, "between", 10, 20), dg.Pred(1, "in", ints=[3000, 3001])], [("pred", 0), ("pred", 1), ("or", 2)]),
        ([dg.Pred(1, "lt", 3000, neg=True), dg.Pred(0, "lt", 2500)], None),
    ]
    for preds, prog in cases:
        for gb in ([0], [1], [1, 0]):
            plan = dg.Plan(preds, gb, aggs, filter=prog)
            ref = oracle_mod.query(table, plan)
            for kernel in (0, 1):
                check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"{preds} {prog} {gb}")


def test_pass_bitmap_predicates_in_clauses(cq, ctx, oracle_mod):
    """Row mode with several RLE / index predicates (pass bitmaps filled once
    per run, complemented for NOT) inside OR clauses, next to predicates on
    plain and packed columns."""
    table, plan = dg.heterogeneous(1_000_003, seed=31)
    c1, c2, c4 = 0, 2, 3                                   # RLE, index, plain
    preds = [dg.Pred(c1, "lt", 300), dg.Pred(c2, "gt", 0), dg.Pred(c4, "between", 100_000, 600_000),
             dg.Pred(c1, "gt", 900), dg.Pred(c2, "eq", 0)]
    progs = [
        [("pred", 0), ("pred", 2), ("or", 2), ("pred", 1), ("not", 0), ("pred", 3), ("or", 2), ("and", 2)],
        [("pred", 0), ("pred", 1), ("and", 2), ("not", 0), ("pred", 4), ("pred", 2), ("and", 2), ("or", 2)],
        [("pred", 3), ("not", 0), ("pred", 4), ("not", 0), ("and", 2), ("pred", 0), ("or", 2)],
    ]
    for prog in progs:
        p = dg.Plan(preds, plan.group_by, plan.aggs, filter=prog)
        ref = oracle_mod.query(table, p, n_threads=4)
        for kernel in (0, 1):
            check(run(cq, ctx, table, p, cq.exec_options(kernel=kernel)), ref, f"{prog} kernel {kernel}")


def test_filters_in_a_batch(cq, ctx, oracle_mod):
    """Queries with programs and OR groups inside one batched launch."""
    rng = np.random.default_rng(515)
    tables, plans, refs, handles = [], [], [], []
    for i in range(12):
        n = int(rng.choice([4000, 30000, 90001]))
        cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(3)]
        table = dg.Table(cols, n)
        plan = with_filter(rng, random_plan(rng, table, n_preds=int(rng.integers(1, 5))), i % 2 == 0)
        t, c = cq.table_from(ctx, table)
        tables.append(t)
        handles.append(c)
        plans.append(plan)
        refs.append(oracle_mod.query(table, plan))
    for i, res in enumerate(cq.cq_batch_run(tables, plans)):
        check(cq.fetch_all(res), refs[i], f"batch query {i}")


def test_filters_through_the_serving_loop(cq, ctx, oracle_mod):
    """The server copies a submitted plan, its filter program included."""
    rng = np.random.default_rng(616)
    srv = cq.cq_server_create(ctx, cq.server_options(max_batch=8))
    table, plan = dg.heterogeneous(300_000, seed=61)
    t, cols = cq.table_from(ctx, table)
    jobs = []
    for i in range(10):
        p = with_filter(rng, random_plan(rng, table, n_preds=int(rng.integers(1, 5)), n_gb=1), i % 2 == 0)
        jobs.append((cq.cq_server_submit(srv, t, p), p))
    for ticket, p in jobs:
        res, _ = cq.cq_server_wait(srv, ticket)
        check(cq.fetch_all(res), oracle_mod.query(table, p, n_threads=4), f"ticket {ticket}")
