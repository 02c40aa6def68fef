"""Pins of the oracle's VAR and STD (Section 7: computed from COUNT, SUM and
the sum of squares).  The oracle forms the exact numerator n * S2 - S1^2 in
256-bit integers and rounds the quotient once; the pins are closed forms,
Python's exact rationals (Fraction -> float rounds correctly), the numpy
formulation over random tables, and invariances (shift, weighting by runs,
chunked scans)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests import tensor_ref
from tests.helpers import random_column, random_plan
from tests.test_oracle import assert_same

VAR_OPS = ("var_pop", "var_samp", "std_pop", "std_samp")


def aggs_of(col):
    return [dg.Agg(op, col) for op in VAR_OPS] + [dg.Agg("count")]


def exact(values, op):
    n = len(values)
    d = n - (1 if op.endswith("samp") else 0)
    if n == 0 or d == 0:
        return 0.0
    s1, s2 = sum(values), sum(x * x for x in values)
    v = float(Fraction(n * s2 - s1 * s1, n * d))
    return math.sqrt(v) if op.startswith("std") else v


@pytest.mark.parametrize("n", [1, 2, 3, 10, 97, 1000, 65537])
def test_closed_form_of_consecutive_integers(oracle_mod, n):
    """1..n: the population variance is (n^2 - 1) / 12, the sample variance
    n (n + 1) / 12."""
    t = dg.Table([dg.Plain(np.arange(1, n + 1, dtype=np.int64))], n)
    o = oracle_mod.query(t, dg.Plan([], [], aggs_of(0)))
    assert o.aggs[0][0] == float(Fraction(n * n - 1, 12))
    assert o.aggs[1][0] == (float(Fraction(n * (n + 1), 12)) if n > 1 else 0.0)
    assert o.aggs[2][0] == math.sqrt(float(Fraction(n * n - 1, 12)))


def test_constant_two_values_and_empty(oracle_mod):
    n = 1001
    t = dg.Table([dg.Plain(np.full(n, -123456789, dtype=np.int64)),
                  dg.Plain(np.array(np.where(np.arange(1000) % 2 == 0, 7, 19).tolist() + [13], dtype=np.int64))], n)
    o = oracle_mod.query(t, dg.Plan([], [], aggs_of(0)))
    assert [float(a[0]) for a in o.aggs[:4]] == [0.0, 0.0, 0.0, 0.0]
    # 500 sevens, 500 nineteens and a 13: the mean is 13, the squared deviations 36
    o = oracle_mod.query(t, dg.Plan([], [], aggs_of(1)))
    assert o.aggs[0][0] == float(Fraction(1000 * 36, 1001)) and o.aggs[1][0] == 36.0
    # nothing passes: no rows, every statistic 0
    o = oracle_mod.query(t, dg.Plan([dg.Pred(0, "gt", 0)], [], aggs_of(1)))
    assert [float(a[0]) for a in o.aggs[:4]] == [0.0] * 4 and int(o.aggs[4][0]) == 0


@pytest.mark.parametrize("seed", range(12))
def test_extreme_values_stay_exact(oracle_mod, seed):
    """Values near +-2^62 and +-2^63: S1^2 and n * S2 exceed 128 bits."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 3000))
    lo, hi = [(-(1 << 63), (1 << 63) - 1), ((1 << 62) - 1000, (1 << 62)), (-(1 << 63), -(1 << 63) + 50)][seed % 3]
    vals = rng.integers(lo, hi, size=n, endpoint=True, dtype=np.int64)
    t = dg.Table([dg.Plain(vals)], n)
    o = oracle_mod.query(t, dg.Plan([], [], aggs_of(0)))
    py = [int(x) for x in vals]
    for i, op in enumerate(VAR_OPS):
        assert o.aggs[i][0] == exact(py, op), op


@pytest.mark.parametrize("seed", range(20))
def test_random_tables_match_tensor_formulation(oracle_mod, seed):
    rng = np.random.default_rng(2200 + seed)
    n = int(rng.integers(1, 400))
    cols = [random_column(rng, n, str(rng.choice(["rle", "plain", "packed", "index"]))) for _ in range(3)]
    t = dg.Table(cols, n)
    plan = random_plan(rng, t, allow=("sum", "count", "min", "max") + VAR_OPS)
    assert_same(oracle_mod.query(t, plan), tensor_ref.query(t, plan))
    assert_same(oracle_mod.query(t, plan, n_threads=3, row_ranges=[(0, n // 2), (n // 2, n)]),
                tensor_ref.query(t, plan))


def test_shift_invariance_and_run_weighting(oracle_mod):
    """VAR(x + c) = VAR(x) exactly; an RLE column's runs weigh by length."""
    rng = np.random.default_rng(8)
    n = 50_000
    a = dg.make_rle(rng, n, 7.0, -300, 300, np.int64, np.int64)
    flat = np.repeat(a.run_values, np.diff(np.concatenate([[0], a.run_ends])))
    b = dg.RLE(a.run_values + (1 << 40), a.run_ends, n)
    t = dg.Table([a, b, dg.Plain(flat)], n)
    oa = oracle_mod.query(t, dg.Plan([], [], aggs_of(0)))
    ob = oracle_mod.query(t, dg.Plan([], [], aggs_of(1)))
    oc = oracle_mod.query(t, dg.Plan([], [], aggs_of(2)))
    for i, op in enumerate(VAR_OPS):
        assert oa.aggs[i][0] == ob.aggs[i][0] == oc.aggs[i][0] == exact([int(x) for x in flat], op), op


def test_large_chunked_scan(oracle_mod):
    """Several 1M-row chunks merged: the per-chunk sums of squares add up."""
    rng = np.random.default_rng(3)
    n = 2_500_000
    v = rng.integers(-(1 << 31), 1 << 31, size=n).astype(np.int64)
    g = rng.integers(0, 3, size=n).astype(np.int64)
    t = dg.Table([dg.Plain(g), dg.Plain(v)], n)
    o = oracle_mod.query(t, dg.Plan([], [0], aggs_of(1)), n_threads=4)
    for k in range(3):
        part = [int(x) for x in v[g == k]]
        for i, op in enumerate(VAR_OPS):
            assert o.aggs[i][k] == exact(part, op), (k, op)


def test_rounding_of_the_quotient(oracle_mod):
    """The division step against Python's correctly rounded Fraction -> float,
    on cases where only the bits beyond the first 64 of the quotient decide:
    exactly halfway between two doubles, and halfway plus a tiny excess (the
    remainder must break the tie upward), at magnitudes from 2^-100 to 2^200."""
    rng = np.random.default_rng(17)
    cases = []
    for e in (53, 60, 100, 150, 200):
        for d in (1 << 20, 3, 1_000_003, (1 << 127) - 1):
            half = (1 << e) + 1                     # odd at 2^e: halfway between two doubles above 2^53
            for num in (half * d, half * d + 1, half * d - 1):
                if 0 <= num < 1 << 256:
                    cases.append((num, d))
    for _ in range(300):
        d = int(rng.integers(1, 1 << 62)) * int(rng.integers(1, 1 << 62)) + 1
        n = int.from_bytes(rng.bytes(32), "little") >> int(rng.integers(0, 250))
        cases.append((n, d))
    cases.append((1, (1 << 127) + 12345))
    for n, d in cases:
        assert oracle_mod.div_round(n, d) == float(Fraction(n, d)), (n, d)
