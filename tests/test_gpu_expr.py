"""GPU parity for aggregates over position-wise arithmetic of two columns
(Section 6: arithmetic on aligned columns; the paper's c1 + c2 example).
Segment mode evaluates A (op) B once per aligned segment; row mode runs the
generic row kernel.  Covered: the paper's example, every non-dictionary
encoding under both segment walks, row mode, decompress-then-scan, a batch,
products near 2^62 (128-bit sums), and the planner's refusals.  The bar is
bit-exact equality with the CPU oracle."""
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, rle_inclusive

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OPS = ("add", "sub", "mul")


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


def test_paper_example(cq, ctx, oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "aligned_add_example.json")))
    c1 = rle_inclusive(g["c1"]["val"], g["c1"]["start"], g["c1"]["end"])
    c2 = rle_inclusive(g["c2"]["val"], g["c2"]["start"], g["c2"]["end"])
    table = dg.Table([c1, c2], 40)
    plan = dg.Plan([], [0, 1], [dg.Agg("min", 0, "add", 1), dg.Agg("sum", 0, "add", 1), dg.Agg("count")])
    ref = oracle_mod.query(table, plan)
    assert sorted(ref.aggs[0].tolist()) == sorted(g["sum_val"])
    for kernel in (0, 2, 3):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"kernel {kernel}")


@pytest.mark.parametrize("seed", range(16))
def test_segment_mode(cq, ctx, oracle_mod, seed):
    """RLE and index columns only: both segment walks."""
    rng = np.random.default_rng(16000 + seed)
    n = int(rng.choice([3000, 70001, 200003]))
    cols = [random_column(rng, n, str(rng.choice(["rle", "index"])), lo=-(1 << 20), hi=1 << 20) for _ in range(3)]
    cols.append(dg.make_rle(rng, n, 40.0, 0, 12, np.int64, np.int64))
    table = dg.Table(cols, n)
    aggs = [dg.Agg(op, int(rng.integers(0, 3)), str(rng.choice(OPS)), int(rng.integers(0, 3)))
            for op in ("sum", "min", "max", "avg")] + [dg.Agg("count")]
    preds = [dg.Pred(3, "lt", 9)] if seed % 2 else []
    plan = dg.Plan(preds, [3], aggs)
    ref = oracle_mod.query(table, plan)
    for kernel in (2, 3):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


@pytest.mark.parametrize("seed", range(16))
def test_row_mode(cq, ctx, oracle_mod, seed):
    """Every non-dictionary encoding, several tiles and a ragged tail; the
    default (generic row kernel for expressions) and decompress-then-scan."""
    rng = np.random.default_rng(17000 + seed)
    n = int(rng.choice([1, 1000, 20000, 70001]))
    encs = ["rle", "plain", "packed", "index"]
    cols = [random_column(rng, n, str(rng.choice(encs)), lo=-(1 << 20), hi=1 << 20) for _ in range(3)]
    cols.append(random_column(rng, n, "plain", lo=0, hi=7))
    table = dg.Table(cols, n)
    aggs = [dg.Agg(str(rng.choice(["sum", "min", "max", "avg"])), int(rng.integers(0, 3)), str(rng.choice(OPS)),
                   int(rng.integers(0, 3))) for _ in range(4)] + [dg.Agg("count"), dg.Agg("sum", 0)]
    preds = [dg.Pred(int(rng.integers(0, 3)), "between", -(1 << 19), 1 << 19)] if seed % 2 else []
    plan = dg.Plan(preds, [3] if seed % 3 else [], aggs)
    ref = oracle_mod.query(table, plan)
    check(run(cq, ctx, table, plan), ref, f"seed {seed}")
    check(run(cq, ctx, table, plan, cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN)), ref, f"dts {seed}")


def test_products_near_2_62(cq, ctx, oracle_mod):
    """|A|, |B| < 2^31: products near 2^62 (MIN / MAX) and group sums beyond
    2^64 (AVG from 128-bit words)."""
    rng = np.random.default_rng(3)
    n = 400_001
    a = dg.Plain(rng.integers(-(1 << 31) + 1, 1 << 31, size=n).astype(np.int64))
    b = dg.make_packed(rng.integers(0, 1 << 31, size=n).astype(np.uint64), 31, -(1 << 30))
    g = dg.Plain(rng.integers(0, 5, size=n).astype(np.int64))
    table = dg.Table([a, b, g], n)
    plan = dg.Plan([], [2], [dg.Agg("max", 0, "mul", 1), dg.Agg("min", 0, "mul", 1), dg.Agg("avg", 0, "mul", 1)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), "products")


def test_batch_and_refusals(cq, ctx, oracle_mod):
    rng = np.random.default_rng(44)
    tables, plans, refs, keep = [], [], [], []
    for i in range(6):
        n = int(rng.choice([3000, 40001]))
        enc = ["rle", "index"] if i % 2 else ["rle", "plain", "packed", "index"]
        cols = [random_column(rng, n, str(rng.choice(enc)), lo=-5000, hi=5000) for _ in range(3)]
        table = dg.Table(cols, n)
        plan = dg.Plan([], [0], [dg.Agg("sum", 1, str(rng.choice(OPS)), 2), dg.Agg("count"),
                                 dg.Agg("max", 2, "sub", 1)])
        t, c = cq.table_from(ctx, table)
        tables.append(t)
        keep.append(c)
        plans.append(plan)
        refs.append(oracle_mod.query(table, plan))
    for i, res in enumerate(cq.cq_batch_run(tables, plans)):
        check(cq.fetch_all(res), refs[i], f"batch {i}")
    n = 100
    big = dg.Plain(np.full(n, 1 << 40, dtype=np.int64))
    d = dg.make_dict([b"a", b"b"], np.zeros(n, dtype=np.uint64), 1)
    t, cols = cq.table_from(ctx, dg.Table([big, big, d], n))
    with pytest.raises(cq.CQError) as e:     # 2^80 per row
        cq.cq_query_run(t, dg.Plan([], [], [dg.Agg("sum", 0, "mul", 1)]))
    assert e.value.status == cq.CQ_ERR_UNSUPPORTED
    for bad in (dg.Agg("sum", 0, "add", 2), dg.Agg("var_pop", 0, "add", 1)):
        with pytest.raises(cq.CQError) as e:
            cq.cq_query_run(t, dg.Plan([], [], [bad]))
        assert e.value.status == cq.CQ_ERR_INVALID_ARG
