"""Pins of the oracle's aggregates over position-wise arithmetic of two
columns (Section 6, Arithmetic, Comparison, and Selection Operations: align
the columns, then operate on the aligned values).  The pins: the paper's
c1 + c2 example (aligned runs and summed values), linearity identities,
constant operands, exact brute force with Python integers, and the int64
range of a row's result."""
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests import tensor_ref
from tests.helpers import random_column, rle_inclusive
from tests.test_oracle import assert_same

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_columns():
    g = json.load(open(os.path.join(GOLDEN, "aligned_add_example.json")))
    c1 = rle_inclusive(g["c1"]["val"], g["c1"]["start"], g["c1"]["end"])
    c2 = rle_inclusive(g["c2"]["val"], g["c2"]["start"], g["c2"]["end"])
    return g, c1, c2


def test_paper_example(oracle_mod):
    """c1 + c2 on the paper's two RLE columns: grouping by (c1, c2) gives one
    group per aligned segment, whose MIN = MAX = the printed sum, and whose
    COUNT = the segment's length."""
    g, c1, c2 = paper_columns()
    n = 40
    t = dg.Table([c1, c2], n)
    aggs = [dg.Agg("min", 0, "add", 1), dg.Agg("max", 0, "add", 1), dg.Agg("sum", 0, "add", 1), dg.Agg("count")]
    o = oracle_mod.query(t, dg.Plan([], [0, 1], aggs))
    lens = [e - s + 1 for s, e in zip(g["aligned_start"], g["aligned_end"])]
    # groups come out in key order; map them back to the segments
    segs = {(a, b): (v, L) for a, b, v, L in zip(g["r1_val"], g["r2_val"], g["sum_val"], lens)}
    assert len(o.keys[0]) == len(segs)
    for k1, k2, mn, mx, sm, cnt in zip(o.keys[0], o.keys[1], o.aggs[0], o.aggs[1], o.aggs[2], o.aggs[3]):
        v, L = segs[(int(k1), int(k2))]
        assert int(mn) == int(mx) == v
        assert int(sm) == v * L and int(cnt) == L
    # the aligned boundaries are the common refinement of the runs
    ends, _ = oracle_mod.align([c1.run_ends, c2.run_ends], n)
    assert [int(e) - 1 for e in ends] == g["aligned_end"]
    o = oracle_mod.query(t, dg.Plan([], [], [dg.Agg("sum", 0, "add", 1)]))
    assert int(o.aggs[0][0]) == sum(v * L for v, L in zip(g["sum_val"], lens))


@pytest.mark.parametrize("seed", range(12))
def test_linearity_and_constants(oracle_mod, seed):
    """SUM(A + B) = SUM(A) + SUM(B), SUM(A - B) = SUM(A) - SUM(B) per group;
    with B a constant column k: SUM(A * B) = k * SUM(A), MIN(A + B) =
    MIN(A) + k, MAX(A - B) = MAX(A) - k."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(1, 3000))
    encs = ["rle", "plain", "packed", "index"]
    a = random_column(rng, n, str(rng.choice(encs)), lo=-1000, hi=1000)
    b = random_column(rng, n, str(rng.choice(encs)), lo=-1000, hi=1000)
    k = int(rng.integers(-9, 10))
    kc = dg.RLE(np.array([k], dtype=np.int64), np.array([n], dtype=np.int64), n)
    key = random_column(rng, n, "rle", lo=0, hi=5)
    t = dg.Table([a, b, kc, key], n)
    aggs = [dg.Agg("sum", 0, "add", 1), dg.Agg("sum", 0), dg.Agg("sum", 1), dg.Agg("sum", 0, "sub", 1),
            dg.Agg("sum", 0, "mul", 2), dg.Agg("min", 0, "add", 2), dg.Agg("min", 0), dg.Agg("max", 0, "sub", 2),
            dg.Agg("max", 0)]
    o = oracle_mod.query(t, dg.Plan([], [3], aggs))
    s_ab, s_a, s_b, s_amb, s_ak, mn_ak, mn_a, mx_amk, mx_a = [x.astype(object) for x in o.aggs]
    for i in range(len(o.keys[0])):
        assert s_ab[i] == s_a[i] + s_b[i]
        assert s_amb[i] == s_a[i] - s_b[i]
        assert s_ak[i] == k * s_a[i]
        assert mn_ak[i] == mn_a[i] + k and mx_amk[i] == mx_a[i] - k


@pytest.mark.parametrize("seed", range(24))
def test_random_tables_match_tensor_formulation(oracle_mod, seed):
    """Every non-dictionary encoding, random predicates and keys, SUM / MIN /
    MAX / AVG of A + B, A - B, A * B: the oracle against the exact numpy
    formulation (Python integers), whole and in row shards."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 500))
    encs = ["rle", "plain", "packed", "index"]
    cols = [random_column(rng, n, str(rng.choice(encs)), lo=-(1 << 20), hi=1 << 20) for _ in range(4)]
    t = dg.Table(cols, n)
    preds = [dg.Pred(int(rng.integers(0, 4)), "between", -(1 << 19), 1 << 19)] if seed % 2 else []
    aggs = [dg.Agg(str(rng.choice(["sum", "min", "max", "avg"])), int(rng.integers(0, 4)),
                   str(rng.choice(["add", "sub", "mul"])), int(rng.integers(0, 4))) for _ in range(4)]
    plan = dg.Plan(preds, [int(rng.integers(0, 4))] if seed % 3 else [], aggs + [dg.Agg("count")])
    assert_same(oracle_mod.query(t, plan), tensor_ref.query(t, plan))
    assert_same(oracle_mod.query(t, plan, n_threads=3, row_ranges=[(0, n // 3), (n // 3, n)]),
                tensor_ref.query(t, plan))


def test_brute_force_products_near_the_int64_range(oracle_mod):
    """A * B with |A|, |B| near 2^31: products near 2^62, sums beyond 2^64
    (exact in the 128-bit accumulator), against Python integers."""
    rng = np.random.default_rng(9)
    n = 5000
    a = rng.integers(-(1 << 31), 1 << 31, size=n).astype(np.int64)
    b = rng.integers(-(1 << 31), 1 << 31, size=n).astype(np.int64)
    g = rng.integers(0, 3, size=n).astype(np.int64)
    t = dg.Table([dg.Plain(a), dg.Plain(b), dg.Plain(g)], n)
    o = oracle_mod.query(t, dg.Plan([], [2], [dg.Agg("sum", 0, "mul", 1), dg.Agg("max", 0, "mul", 1)]))
    for k in range(3):
        m = g == k
        prods = [int(x) * int(y) for x, y in zip(a[m], b[m])]
        lo, hi = o.sum128[0]
        assert (int(hi[k]) << 64) + int(lo[k]) == sum(prods)
        assert int(o.aggs[1][k]) == max(prods)


def test_results_outside_int64_and_invalid_plans(oracle_mod):
    n = 10
    big = dg.Plain(np.full(n, 1 << 40, dtype=np.int64))
    t = dg.Table([big, big, dg.make_dict([b"a", b"b"], np.zeros(n, dtype=np.uint64), 1)], n)
    with pytest.raises(ValueError, match="status -6"):     # 2^80 per row
        oracle_mod.query(t, dg.Plan([], [], [dg.Agg("sum", 0, "mul", 1)]))
    oracle_mod.query(t, dg.Plan([], [], [dg.Agg("sum", 0, "add", 1)]))   # 2^41 fits
    for bad in (dg.Agg("sum", 0, "add", 2), dg.Agg("var_pop", 0, "add", 1), dg.Agg("sum", 0, "add", 7)):
        with pytest.raises(ValueError, match="status -1"):
            oracle_mod.query(t, dg.Plan([], [], [bad]))
