"""GPU parity for key domains above 2^24 groups (the global hash table of
packed keys, sorted at finalize) and for values and literals at the ends of
the int64 range.  Every result is compared with the CPU oracle element by
element; the bar is bit-exact equality (AVG included)."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column

pytestmark = pytest.mark.gpu

I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1


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


AGGS5 = [dg.Agg("sum", 2), dg.Agg("sum", 4), dg.Agg("min", 4), dg.Agg("max", 4), dg.Agg("count"), dg.Agg("avg", 4),
         dg.Agg("min", 2), dg.Agg("max", 2)]


@pytest.mark.parametrize("kernel", [0, 1])
def test_group_by_rle_key_and_plain_column(cq, ctx, oracle_mod, kernel):
    """GROUP BY c1, c4 on the heterogeneous table: 1000 x 1,000,001 possible
    groups (about 1e9), far above the dense limit."""
    table, plan = dg.heterogeneous(400_000 + 333, seed=11)
    plan = dg.Plan(plan.preds, [0, 3], AGGS5)
    ref = oracle_mod.query(table, plan, n_threads=4)
    assert len(ref.keys[0]) > 1000
    check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)), ref, f"c1,c4 kernel {kernel}")


def test_group_by_index_encoded_int64(cq, ctx, oracle_mod):
    """GROUP BY the index-encoded int64 column (values in +-2^40 and the
    default): a 2^41-value domain."""
    table, plan = dg.heterogeneous(300_001, seed=12, index_default=-7)
    plan = dg.Plan([plan.preds[1]], [2], [dg.Agg("count"), dg.Agg("sum", 4), dg.Agg("min", 3), dg.Agg("avg", 2)])
    ref = oracle_mod.query(table, plan, n_threads=4)
    check(run(cq, ctx, table, plan), ref, "c3")


@pytest.mark.parametrize("lg", [12, 14])
def test_full_table_is_retried_larger(cq, ctx, oracle_mod, lg):
    """A global table far too small for the groups (2^12 or 2^14 slots for
    about 60,000 groups) fills on the device; cq_result_wait relaunches with
    four times the slots until the groups fit, and the result is exact."""
    table, plan = dg.heterogeneous(250_000, seed=13)
    plan = dg.Plan([], [0, 3], [dg.Agg("count"), dg.Agg("sum", 4)])
    ref = oracle_mod.query(table, plan, n_threads=4)
    assert len(ref.keys[0]) > 4 * (1 << lg)
    check(run(cq, ctx, table, plan, cq.exec_options(hash_slots_log2=lg)), ref, f"retry from 2^{lg}")


def test_segment_mode_wide_keys(cq, ctx, oracle_mod):
    """Two RLE columns of wide int64 values (segment mode) grouped together."""
    rng = np.random.default_rng(14)
    n = 200_003
    a = dg.make_rle(rng, n, 5.0, -(1 << 35), 1 << 35, np.int64, np.int64)   # 2^36 x 2^20 key values
    b = dg.make_rle(rng, n, 3.0, 0, 1 << 20, np.int64, np.int64)
    table = dg.Table([a, b], n)
    plan = dg.Plan([dg.Pred(1, "lt", 1 << 19)], [0, 1], [dg.Agg("sum", 1), dg.Agg("count"), dg.Agg("max", 0)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), "segment wide")


@pytest.mark.parametrize("seed", range(16))
def test_random_wide_tables(cq, ctx, oracle_mod, seed):
    """Random tables of every encoding with values spread over +-2^40,
    +-2^15 and +-2^18, one or two group-by columns (hash domains of up to
    about 2^60 groups), random predicates."""
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.choice([1000, 4097, 50001]))
    encs = ["rle", "plain", "index", "packed"]
    cols = [random_column(rng, n, str(rng.choice(encs)), lo=-(1 << b), hi=1 << b) for b in (40, 15, 18)]
    table = dg.Table(cols, n)
    gb = list(rng.choice(3, size=int(rng.integers(1, 3)), replace=False))
    preds = []
    if rng.random() < 0.7:
        c = int(rng.integers(0, 3))
        b = (40, 15, 18)[c]
        lo = int(rng.integers(-(1 << b), 1 << b))
        preds.append(dg.Pred(c, "between", lo, lo + (1 << (b - 1))))
    aggs = [dg.Agg("count"), dg.Agg("sum", int(rng.integers(0, 3))), dg.Agg("min", int(rng.integers(0, 3))),
            dg.Agg("max", int(rng.integers(0, 3))), dg.Agg("avg", int(rng.integers(0, 3)))]
    plan = dg.Plan(preds, [int(g) for g in gb], aggs)
    ref = oracle_mod.query(table, plan)
    check(run(cq, ctx, table, plan), ref, f"seed {seed}")


def _extreme_column(rng, n, enc, lo, hi):
    vals = rng.integers(lo, hi, size=n, endpoint=True, dtype=np.int64)
    if enc == "plain":
        return dg.Plain(vals)
    if enc == "rle":
        ends = dg.geometric_ends(rng, n, 4.0, np.int64)
        return dg.RLE(rng.integers(lo, hi, size=ends.shape[0], endpoint=True, dtype=np.int64), ends, n)
    nnz = n // 3
    pos = np.sort(rng.choice(n, size=nnz, replace=False)).astype(np.int64)
    return dg.Index(vals[:nnz], pos, int(lo), n)


@pytest.mark.parametrize("enc", ["plain", "rle", "index"])
def test_int64_extreme_values_and_literals(cq, ctx, oracle_mod, enc):
    """Key values near INT64_MAX and INT64_MIN (so the key minimum sits at the
    edge of the range), predicates with literals at INT64_MIN / INT64_MAX,
    MIN / MAX over extreme values, and COUNT."""
    rng = np.random.default_rng(99)
    n = 20_011
    k_hi = _extreme_column(rng, n, enc, I64_MAX - 500, I64_MAX)
    k_lo = _extreme_column(rng, n, enc, I64_MIN, I64_MIN + 300)
    v = _extreme_column(rng, n, enc, I64_MIN, I64_MAX)
    table = dg.Table([k_hi, k_lo, v], n)
    aggs = [dg.Agg("count"), dg.Agg("min", 2), dg.Agg("max", 2), dg.Agg("min", 0), dg.Agg("max", 1)]
    for preds in ([dg.Pred(2, "le", I64_MAX), dg.Pred(0, "ge", I64_MIN)],
                  [dg.Pred(2, "between", I64_MIN, I64_MAX)],
                  [dg.Pred(0, "gt", I64_MAX - 250), dg.Pred(1, "lt", I64_MIN + 150)],
                  [dg.Pred(2, "lt", I64_MIN)],
                  [dg.Pred(2, "gt", I64_MAX)],
                  [dg.Pred(1, "ne", I64_MIN), dg.Pred(0, "eq", I64_MAX)]):
        for gb in ([0], [1], [0, 1]):
            plan = dg.Plan(preds, gb, aggs)
            check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), f"{enc} {preds} {gb}")


def test_extreme_sums_overflow_like_the_oracle(cq, ctx, oracle_mod):
    """SUM over values near the int64 bounds: the exact 128-bit sum does not
    fit int64, the oracle's status says so, and the library reports
    CQ_ERR_OVERFLOW."""
    rng = np.random.default_rng(5)
    n = 10_000
    key = dg.Plain(rng.integers(0, 50, size=n).astype(np.int64))
    big = dg.Plain(rng.integers(I64_MAX - (1 << 20), I64_MAX, size=n, endpoint=True, dtype=np.int64))
    table = dg.Table([key, big], n)
    plan = dg.Plan([], [0], [dg.Agg("sum", 1), dg.Agg("count")])
    ref = oracle_mod.query(table, plan)
    assert ref.status != 0
    t, cols = cq.table_from(ctx, table)
    res = cq.cq_query_run(t, plan)
    with pytest.raises(cq.CQError) as e:
        cq.cq_result_wait(res)
    assert e.value.status == cq.CQ_ERR_OVERFLOW


@pytest.mark.parametrize("rows", [65536, 200_000])
def test_split_launches_fold_the_sums(cq, ctx, oracle_mod, rows):
    """A query over more rows than one launch takes runs as several launches
    with the SUM limb words folded in between (normally above 2^31 rows;
    CQ_LAUNCH_ROWS lowers the split here).  Results stay exact, for the
    specialised and the generic kernel and in segment mode."""
    import os
    table, plan = dg.heterogeneous(1_000_003, seed=21)
    tiny, tplan = dg.tiny_two_rle(700_001, seed=22)
    old = os.environ.get("CQ_LAUNCH_ROWS")
    os.environ["CQ_LAUNCH_ROWS"] = str(rows)
    try:
        for kernel in (0, 1):
            check(run(cq, ctx, table, plan, cq.exec_options(kernel=kernel)),
                  oracle_mod.query(table, plan, n_threads=4), f"split {rows} kernel {kernel}")
        check(run(cq, ctx, tiny, tplan), oracle_mod.query(tiny, tplan), f"split {rows} segment mode")
    finally:
        if old is None:
            del os.environ["CQ_LAUNCH_ROWS"]
        else:
            os.environ["CQ_LAUNCH_ROWS"] = old
