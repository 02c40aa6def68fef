"""GPU parity for the RLE + Index composite encoding (Section 3.2: RLE runs
for pure stretches, Index entries for scattered rows).  The library merges
the two parts into one RLE column at creation; queries on it must equal the
CPU oracle, which decodes the composite itself.  Covered: the paper's
example, random compositions in row mode (specialised and generic kernels)
and segment mode (both walks), predicates, keys and aggregates on composite
columns, the merged column's size, and the rejection of gaps, overlaps and
empty runs."""
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, random_plan
from tests.test_oracle_composite import letters, random_sequence

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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
    g = json.load(open(os.path.join(GOLDEN, "rle_index_example.json")))
    n = len(g["sequence"])
    col = dg.RLEIndex(np.array(letters(g["rle"]["v"]), np.int64), np.array(g["rle"]["s"], np.int64),
                      np.array(g["rle"]["e"], np.int64) + 1, np.array(letters(g["index"]["v"]), np.int64),
                      np.array(g["index"]["p"], np.int64), n)
    table = dg.Table([col, dg.Plain(np.arange(n, dtype=np.int64))], n)
    plan = dg.Plan([], [0], [dg.Agg("count"), dg.Agg("sum", 1), dg.Agg("min", 1)])
    ref = oracle_mod.query(table, plan)
    assert ref.keys[0].tolist() == sorted(set(letters(g["sequence"])))
    check(run(cq, ctx, table, plan), ref, "row mode")
    h = cq.column_from(ctx, col)
    assert cq.cq_column_encoding(h) == 1
    assert cq.cq_column_device_bytes(h) == 4 * 8 + 4 * 4      # 4 runs: int64 values, int32 ends


@pytest.mark.parametrize("seed", range(16))
def test_random_compositions(cq, ctx, oracle_mod, seed):
    rng = np.random.default_rng(18000 + seed)
    n = int(rng.choice([1, 1000, 20000, 70001]))
    cols = [dg.rle_index_encode(random_sequence(rng, n), int(rng.integers(1, 10))) for _ in range(2)]
    other = str(rng.choice(["plain", "packed", "rle", "index"]))
    cols.append(random_column(rng, n, other))
    table = dg.Table(cols, n)
    plan = random_plan(rng, dg.Table([dg.Plain(random_sequence(rng, n)) for _ in range(3)], n))
    plan = dg.Plan([dg.Pred(int(p.col), p.op, p.lo, p.hi, ints=p.ints, group=p.group, neg=p.neg) for p in plan.preds
                    if p.strs is None], plan.group_by, [a for a in plan.aggs])
    ref = oracle_mod.query(table, plan)
    kernels = (0, 1, 2, 3) if other in ("rle", "index") else (0, 1)
    for kernel in kernels:
        check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")


def test_rejections(cq, ctx):
    def make(rv, rs, re_, v, p, n):
        return cq.cq_column_create_rle_index(ctx, np.array(rv, np.int64), np.array(rs, np.int64),
                                             np.array(re_, np.int64), np.array(v, np.int64), np.array(p, np.int64), n)
    make([1, 2], [0, 5], [3, 8], [7, 9], [3, 4], 8)
    for args in (([1, 2], [0, 5], [3, 8], [7], [3], 8),          # row 4 uncovered
                 ([1, 2], [0, 4], [5, 8], [7], [4], 8),          # row 4 covered twice
                 ([1, 2], [0, 5], [3, 8], [7, 9], [3, 4], 9),    # coverage 8 of 9
                 ([1, 2], [5, 0], [8, 3], [7, 9], [3, 4], 8)):   # runs out of order
        with pytest.raises(cq.CQError) as e:
            make(*args)
        assert e.value.status == cq.CQ_ERR_SIZE_MISMATCH
    with pytest.raises(cq.CQError) as e:                          # an empty run
        make([1, 2, 3], [0, 3, 3], [3, 3, 8], [], [], 8)
    assert e.value.status == cq.CQ_ERR_UNSORTED
