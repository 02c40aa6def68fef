"""GPU parity for VAR and STD (Section 7: from COUNT, SUM and the sum of
squares; population and sample forms).  The library keeps exact sums of the
values and of their squares (shifted by the packed base or the index
default, which leaves a variance unchanged) and rounds the exact quotient
once at finalize, as the oracle does, so the bar is bit-exact equality."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, random_plan

pytestmark = pytest.mark.gpu

VAR_OPS = ("var_pop", "var_samp", "std_pop", "std_samp")


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


@pytest.mark.parametrize("seed", range(24))
def test_random_tables(cq, ctx, oracle_mod, seed):
    """Every encoding, one or two group-by columns, random predicates, VAR
    and STD beside the other aggregates; specialised and generic kernels."""
    rng = np.random.default_rng(14000 + seed)
    n = int(rng.choice([1, 1000, 4097, 20000, 70001]))
    cols = [random_column(rng, n, str(rng.choice(["rle", "plain", "packed", "index"]))) for _ in range(3)]
    table = dg.Table(cols, n)
    plan = random_plan(rng, table, allow=("sum", "count", "min", "max", "avg") + VAR_OPS)
    plan = dg.Plan(plan.preds, plan.group_by,
                   plan.aggs + [dg.Agg(str(rng.choice(VAR_OPS)), int(rng.integers(0, 3)))])
    ref = oracle_mod.query(table, plan)
    for kernel in (0, 1):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


@pytest.mark.parametrize("seed", range(8))
def test_segment_mode(cq, ctx, oracle_mod, seed):
    """RLE / index columns only: squares weighted by segment length, walking
    tiles and runs."""
    rng = np.random.default_rng(15000 + seed)
    n = int(rng.choice([5000, 200_001]))
    cols = [random_column(rng, n, str(rng.choice(["rle", "index"])), lo=-(1 << 30), hi=1 << 30) for _ in range(2)]
    cols.append(dg.make_rle(rng, n, 50.0, 0, 20, np.int64, np.int64))
    table = dg.Table(cols, n)
    plan = dg.Plan([], [2], [dg.Agg(op, 0) for op in VAR_OPS] + [dg.Agg("var_samp", 1), dg.Agg("std_pop", 1),
                             dg.Agg("count")])
    ref = oracle_mod.query(table, plan)
    for kernel in (2, 3):
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


def test_extreme_inputs(cq, ctx, oracle_mod):
    """Values at +-(2^31 - 1), a packed column with a base of 2^40 and 20-bit
    offsets, an index column whose default lies 2^40 away from zero, long
    runs (squares times lengths above 2^64), and a single group of 3M rows."""
    rng = np.random.default_rng(77)
    n = 1_000_001
    a = dg.Plain(rng.choice([-(1 << 31) + 1, (1 << 31) - 1, 0, 5], size=n).astype(np.int64))
    b = dg.make_packed(rng.integers(0, 1 << 20, size=n).astype(np.uint64), 20, 1 << 40)
    pos = np.sort(rng.choice(n, size=n // 50, replace=False)).astype(np.int64)
    c = dg.Index((1 << 40) + rng.integers(-(1 << 30), 1 << 30, size=pos.shape[0]).astype(np.int64), pos,
                 1 << 40, n)
    d = dg.make_rle(rng, n, 50_000.0, -(1 << 31) + 1, (1 << 31) - 1, np.int64, np.int64)
    k = dg.Plain(rng.integers(0, 3, size=n).astype(np.int64))
    table = dg.Table([a, b, c, d, k], n)
    aggs = [dg.Agg(op, col) for op in VAR_OPS for col in range(4)]   # 16 aggregates with their companions
    aggs = aggs[:8]
    for gb in ([], [4]):
        plan = dg.Plan([], gb, aggs)
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"gb {gb}")
        plan = dg.Plan([], gb, [dg.Agg(op, col) for op in VAR_OPS[2:] for col in range(4)])
        check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"gb {gb} std")


def test_heterogeneous_table(cq, ctx, oracle_mod):
    """The heterogeneous query's groups (run lines on c1) with VAR / STD of
    the plain and the packed column."""
    table, plan = dg.heterogeneous(1_000_003, seed=9)
    p = dg.Plan(plan.preds, plan.group_by,
                [dg.Agg("var_pop", 3), dg.Agg("std_samp", 4), dg.Agg("count"), dg.Agg("avg", 4)])
    check(run(cq, ctx, table, p), oracle_mod.query(table, p, n_threads=4), "het")


def test_unsupported_and_invalid(cq, ctx):
    n = 1000
    big = dg.Plain(np.arange(n, dtype=np.int64) * (1 << 30))       # reaches 2^39
    table = dg.Table([big, dg.Plain(np.arange(n, dtype=np.int64))], n)
    t, cols = cq.table_from(ctx, table)
    with pytest.raises(cq.CQError) as e:
        cq.cq_query_run(t, dg.Plan([], [], [dg.Agg("var_pop", 0)]))
    assert e.value.status == cq.CQ_ERR_UNSUPPORTED
    with pytest.raises(cq.CQError) as e:   # 9 VARs and their 9 companions exceed 16 aggregates
        cq.cq_query_run(t, dg.Plan([], [], [dg.Agg("var_pop", 1)] * 9))
    assert e.value.status == cq.CQ_ERR_INVALID_ARG


def test_in_a_batch(cq, ctx, oracle_mod):
    rng = np.random.default_rng(31)
    tables, plans, refs, keep = [], [], [], []
    for i in range(6):
        n = int(rng.choice([3000, 40001]))
        cols = [random_column(rng, n, str(rng.choice(["rle", "plain", "packed", "index"]))) for _ in range(3)]
        table = dg.Table(cols, n)
        plan = dg.Plan([], [0], [dg.Agg(str(rng.choice(VAR_OPS)), 1), dg.Agg("count"), dg.Agg("std_pop", 2)])
        t, c = cq.table_from(ctx, table)
        tables.append(t)
        keep.append(c)
        plans.append(plan)
        refs.append(oracle_mod.query(table, plan))
    for i, res in enumerate(cq.cq_batch_run(tables, plans)):
        check(cq.fetch_all(res), refs[i], f"batch {i}")
