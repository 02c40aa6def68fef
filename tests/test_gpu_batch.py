"""Batched launches: many queries over partitions of uneven size in one
persistent launch.  Each query's result inside a batch must equal its
one-query result and the oracle's, bit for bit, whatever the batch shape
(tile rows, work items per CTA) and whatever else shares the launch."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, random_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


@pytest.fixture(scope="module")
def ctx(cq):
    return cq.cq_ctx_create(0)


def check(got, ref, msg=""):
    want = ref.keys + ref.aggs
    assert len(got) == len(want), msg
    for i, (g, w) in enumerate(zip(got, want)):
        assert g.dtype == w.dtype, (msg, i)
        np.testing.assert_array_equal(g, w, err_msg=f"{msg} output column {i}")


def same(a, b, msg=""):
    assert len(a) == len(b), msg
    for i, (x, y) in enumerate(zip(a, b)):
        assert x.dtype == y.dtype and np.array_equal(x, y), f"{msg} column {i}"


@pytest.fixture(scope="module")
def pool(cq, ctx):
    """Partitions of both templates at sizes from one row to 1.5M rows."""
    sizes = [1, 777, 4096, 9001, 60_000, 250_000, 1_500_000]
    parts = []
    for i, n in enumerate(sizes):
        tiny, _ = dg.tiny_two_rle(n, seed=100 + i)
        nest, _ = dg.nested(n, seed=200 + i, lean=True)
        parts.append({"n": n, "tiny": (tiny,) + tuple(cq.table_from(ctx, tiny)),
                      "nested": (nest,) + tuple(cq.table_from(ctx, nest, device=bool(i % 2)))})
    return parts


def workload(rng, pool, n_queries):
    qs = dg.batch_queries(rng, n_queries, len(pool))
    tabs, handles, plans = [], [], []
    for part, kind, plan in qs:
        host, handle, _ = pool[part][kind]
        tabs.append(host)
        handles.append(handle)
        plans.append(plan)
    return tabs, handles, plans


@pytest.mark.parametrize("tile,ipc", [(0, 0), (4096, 1), (8192, 8), (4096, 2), (8192, 4)])
def test_batch_equals_solo_and_oracle(cq, ctx, pool, oracle_mod, tile, ipc):
    rng = np.random.default_rng(11 + tile + ipc)
    tabs, handles, plans = workload(rng, pool, 40)
    opts = cq.exec_options(tile_rows=tile, items_per_cta=ipc) if (tile or ipc) else None
    res = cq.cq_batch_run(handles, plans, opts=opts)
    for i, r in enumerate(res):
        got = cq.fetch_all(r)
        check(got, oracle_mod.query(tabs[i], plans[i]), f"query {i}")
        same(got, cq.fetch_all(cq.cq_query_run(handles[i], plans[i])), f"solo {i}")


def test_batch_random_tables_and_plans(cq, ctx, oracle_mod):
    """Every encoding and plan shape the one-query tests use, in one batch."""
    rng = np.random.default_rng(77)
    encs = ["rle", "plain", "packed", "index", "dict"]
    tabs, handles, plans, keep = [], [], [], []
    for _ in range(48):
        n = int(rng.choice([1, 31, 1000, 4097, 20000, 70001]))
        cols = [random_column(rng, n, str(rng.choice(encs))) for _ in range(int(rng.integers(1, 5)))]
        table = dg.Table(cols, n)
        t, c = cq.table_from(ctx, table)
        keep.append(c)
        tabs.append(table)
        handles.append(t)
        plans.append(random_plan(rng, table))
    res = cq.cq_batch_run(handles, plans, opts=cq.exec_options(items_per_cta=2))
    for i, r in enumerate(res):
        check(cq.fetch_all(r), oracle_mod.query(tabs[i], plans[i]), f"query {i}")


def test_graph_replays_keep_earlier_results(cq, ctx, pool, oracle_mod):
    """Batches that reuse one launch graph: results of an earlier batch stay
    valid after later batches have run through the same graph."""
    rng = np.random.default_rng(5)
    runs = []
    for _ in range(4):
        tabs, handles, plans = workload(rng, pool, 16)
        runs.append((tabs, plans, cq.cq_batch_run(handles, plans)))
    for k, (tabs, plans, res) in enumerate(runs):
        for i, r in enumerate(res):
            check(cq.fetch_all(r), oracle_mod.query(tabs[i], plans[i]), f"batch {k} query {i}")


def test_single_query_batch_and_large_batch(cq, ctx, pool, oracle_mod):
    rng = np.random.default_rng(9)
    tabs, handles, plans = workload(rng, pool, 1)
    check(cq.fetch_all(cq.cq_batch_run(handles, plans)[0]), oracle_mod.query(tabs[0], plans[0]), "one")
    tabs, handles, plans = workload(rng, pool, 1024)
    res = cq.cq_batch_run(handles, plans)
    for i in rng.choice(len(res), size=64, replace=False):
        check(cq.fetch_all(res[i]), oracle_mod.query(tabs[i], plans[i]), f"query {i}")


def test_bad_query_rejects_the_batch(cq, ctx, pool):
    rng = np.random.default_rng(3)
    tabs, handles, plans = workload(rng, pool, 6)
    plans[4] = dg.Plan([dg.Pred(99, "lt", 1)], [], [dg.Agg("count")])
    with pytest.raises(cq.CQError) as e:
        cq.cq_batch_run(handles, plans)
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
    assert "batch query 4" in str(e.value)


def test_autotuner_choice_is_used_and_exact(cq, ctx, pool, oracle_mod):
    rng = np.random.default_rng(21)
    tabs, handles, plans = workload(rng, pool, 64)
    best, us = cq.cq_batch_tune(handles, plans)
    assert us > 0
    assert best.tile_rows in (4096, 8192) and best.items_per_cta in (1, 2, 4, 8)
    res = cq.cq_batch_run(handles, plans)     # no options: the tuned shape
    for i, r in enumerate(res):
        check(cq.fetch_all(r), oracle_mod.query(tabs[i], plans[i]), f"query {i}")


def test_repeated_mixed_batches_are_exact(cq, ctx, pool, oracle_mod):
    """Twenty replays of one mixed batch: every result exact every time (a
    race between warps building one column's tile bitmap once showed up
    here as rare, timing-dependent wrong counts)."""
    rng = np.random.default_rng(4096 + 2 + 11)
    tabs, handles, plans = workload(rng, pool, 40)
    refs = [oracle_mod.query(t, p) for t, p in zip(tabs, plans)]
    opts = cq.exec_options(tile_rows=4096, items_per_cta=2)
    for rep in range(20):
        for i, r in enumerate(cq.cq_batch_run(handles, plans, opts=opts)):
            check(cq.fetch_all(r), refs[i], f"replay {rep} query {i}")


def test_batch_rejects_small_tiles(cq, ctx, pool):
    rng = np.random.default_rng(12)
    tabs, handles, plans = workload(rng, pool, 4)
    with pytest.raises(cq.CQError) as e:
        cq.cq_batch_run(handles, plans, opts=cq.exec_options(tile_rows=2048))
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
