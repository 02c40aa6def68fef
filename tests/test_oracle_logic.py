"""Pins of the oracle's logical operators on masks (Section 5: AND, OR, NOT;
Appendix A.1: NOT of an RLE and of an Index mask).

Expected values come from the paper's printed examples (tests/golden, each
with its citation), set algebra over explicit row sets, closed forms
(inclusion-exclusion, complements) and Boolean identities (De Morgan,
distribution, double negation) that relate differently shaped filters to
each other.  Rows a filter keeps are read back exactly by grouping on a
plain row-id column.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests import tensor_ref
from tests.helpers import as_plain, mask_rle, random_column, random_or_groups, random_plan, random_tree
from tests.test_oracle import assert_same

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COUNT = dg.Agg("count")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def kept_rows(oracle_mod, table, preds, filt=None):
    """Rows the filter keeps: the table gets a row-id column appended and
    the query groups by it."""
    n = table.n_rows
    t = dg.Table(list(table.columns) + [as_plain(np.arange(n))], n)
    o = oracle_mod.query(t, dg.Plan(preds, [len(table.columns)], [COUNT], filter=filt))
    assert o.status == 0 and set(o.aggs[0].tolist()) <= {1}
    return o.keys[0].tolist()


def set_algebra(prog, pred_rows, n):
    """Rows of a postfix filter by set operations: NOT is the complement in
    range(n), AND the intersection, OR the union."""
    universe = set(range(n))
    st = []
    for kind, arg in prog:
        if kind == "pred":
            st.append(set(pred_rows[arg]))
        elif kind == "not":
            st.append(universe - st.pop())
        else:
            top = [st.pop() for _ in range(arg)]
            acc = top[0]
            for x in top[1:]:
                acc = (acc & x) if kind == "and" else (acc | x)
            st.append(acc)
    assert len(st) == 1
    return st[0]


def pred_rows(table, p):
    """Rows a single predicate keeps, from the numpy formulation's mask."""
    col = table.columns[p.col]
    return set(np.flatnonzero(tensor_ref._pred_mask(col, tensor_ref.decode(col), p)).tolist())


# ---------------------------------------------------------------- printed examples
def test_not_examples_by_negation(oracle_mod):
    """Appendix A.1: NOT of the RLE mask [0-1],[4-6] over 8 rows keeps
    [2-3],[7]; NOT of the Index mask {2, 5} keeps [0-1],[3-4],[6-7].  Both
    forms of NOT (a negated predicate and a NOT node) give those rows."""
    g = load("not_examples.json")
    r = g["not_rle"]
    n = r["total_size"]
    m = mask_rle(list(zip(r["s"], r["e"])), n)
    want = [i for s, e in zip(r["result_s"], r["result_e"]) for i in range(s, e + 1)]
    t = dg.Table([m], n)
    assert kept_rows(oracle_mod, t, [dg.Pred(0, "eq", 1, neg=True)]) == want
    assert kept_rows(oracle_mod, t, [dg.Pred(0, "eq", 1)], [("pred", 0), ("not", 0)]) == want
    r = g["not_index"]
    n = r["total_size"]
    x = dg.Index(np.ones(len(r["p"]), dtype=np.int64), np.array(r["p"], dtype=np.int64), 0, n)
    want = [i for s, e in zip(r["result_s"], r["result_e"]) for i in range(s, e + 1)]
    t = dg.Table([x], n)
    assert kept_rows(oracle_mod, t, [dg.Pred(0, "eq", 1, neg=True)]) == want
    assert kept_rows(oracle_mod, t, [dg.Pred(0, "eq", 1)], [("pred", 0), ("not", 0)]) == want


def test_or_of_plain_masks_example(oracle_mod):
    """Section 5.2: [T, F, T, F] OR [T, T, F, F] is [T, T, T, F], as an OR
    group and as an OR node."""
    g = load("or_plain_example.json")
    n = len(g["result"])
    t = dg.Table([as_plain(np.array(g["m1"], dtype=np.int64)), as_plain(np.array(g["m2"], dtype=np.int64))], n)
    want = [i for i, x in enumerate(g["result"]) if x]
    grouped = [dg.Pred(0, "eq", 1, group=1), dg.Pred(1, "eq", 1, group=1)]
    assert kept_rows(oracle_mod, t, grouped) == want
    plain = [dg.Pred(0, "eq", 1), dg.Pred(1, "eq", 1)]
    assert kept_rows(oracle_mod, t, plain, [("pred", 0), ("pred", 1), ("or", 2)]) == want
    # and the AND of the same masks (Section 5.1) keeps their intersection
    assert kept_rows(oracle_mod, t, plain) == [i for i in range(n) if g["m1"][i] and g["m2"][i]]


def test_range_union_of_rle_masks(oracle_mod):
    """Section 5.2, RLE OR RLE (range_union): the range-intersection
    example's masks [2-7] and [1-3],[4-5],[6-8] over 9 rows; their union is
    [1-8]."""
    g = load("range_intersect_example.json")
    n = g["n_rows"]
    m1 = mask_rle(list(zip(g["c1"]["start"], g["c1"]["end"])), n)
    m2 = mask_rle(list(zip(g["c2"]["start"], g["c2"]["end"])), n)
    t = dg.Table([m1, m2], n)
    want = set()
    for s, e in zip(g["c1"]["start"] + g["c2"]["start"], g["c1"]["end"] + g["c2"]["end"]):
        want |= set(range(s, e + 1))
    got = kept_rows(oracle_mod, t, [dg.Pred(0, "eq", 1, group=7), dg.Pred(1, "eq", 1, group=7)])
    assert got == sorted(want) == list(range(1, 9))


@pytest.mark.parametrize("seed", range(6))
def test_or_across_encodings_is_the_union(oracle_mod, seed):
    """Section 5.2's cases (RLE OR RLE, RLE OR Index, Index OR Index, with
    Plain) on random masks: the kept rows are the union of the row sets."""
    rng = np.random.default_rng(40 + seed)
    n = int(rng.integers(20, 200))

    def rle_mask():
        cuts = np.sort(rng.choice(np.arange(1, n), size=int(rng.integers(0, min(n - 1, 12))), replace=False))
        ends = np.concatenate([cuts, [n]]).astype(np.int64)
        vals = rng.integers(0, 2, size=ends.shape[0]).astype(np.int64)
        return dg.RLE(vals, ends, n)

    def idx_mask():
        pos = np.sort(rng.choice(n, size=int(rng.integers(0, n // 3 + 1)), replace=False)).astype(np.int64)
        return dg.Index(np.ones(pos.shape[0], dtype=np.int64), pos, 0, n)

    cols = [rle_mask(), rle_mask(), idx_mask(), idx_mask(), as_plain(rng.integers(0, 2, size=n))]
    t = dg.Table(cols, n)
    sets = [pred_rows(t, dg.Pred(c, "eq", 1)) for c in range(5)]
    for a, b in itertools.combinations(range(5), 2):
        got = kept_rows(oracle_mod, t, [dg.Pred(a, "eq", 1, group=3), dg.Pred(b, "eq", 1, group=3)])
        assert got == sorted(sets[a] | sets[b]), (a, b)


# ---------------------------------------------------------------- closed forms and identities
def _random_atoms(rng, n, k):
    cols = [random_column(rng, n, str(rng.choice(["rle", "plain", "packed", "index", "dict"]))) for _ in range(3)]
    t = dg.Table(cols, n)
    return t, random_plan(rng, t, n_preds=k, n_gb=1).preds


@pytest.mark.parametrize("seed", range(12))
def test_inclusion_exclusion_and_complement(oracle_mod, seed):
    """|a OR b| = |a| + |b| - |a AND b| and |NOT a| = n - |a|."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 400))
    t, (a, b) = _random_atoms(rng, n, 2)

    def count(preds, filt=None):
        return int(oracle_mod.query(t, dg.Plan(preds, [], [COUNT], filter=filt)).aggs[0][0])

    both = count([a, b])
    either = count([a, b], [("pred", 0), ("pred", 1), ("or", 2)])
    assert either == count([a]) + count([b]) - both
    assert count([a], [("pred", 0), ("not", 0)]) == n - count([a])
    assert count([dataclasses_replace(a, neg=True)]) == n - count([a])


def dataclasses_replace(p, **kw):
    import dataclasses
    return dataclasses.replace(p, **kw)


@pytest.mark.parametrize("seed", range(12))
def test_boolean_identities(oracle_mod, seed):
    """De Morgan (the composite-mask rewrites of Section 5.3), distribution
    of AND over OR, double negation: both sides give identical results,
    aggregates included, in program form and in OR-group form."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 300))
    t, (a, b, c) = _random_atoms(rng, n, 3)
    plan = random_plan(rng, t, n_preds=0, n_gb=1)
    P, A, B, Cn, N = ("pred", 0), ("pred", 1), ("pred", 2), ("not", 0), None

    def q(preds, filt=N):
        return oracle_mod.query(t, dg.Plan(preds, plan.group_by, plan.aggs, filter=filt))

    def same(x, y):
        assert len(x.keys) == len(y.keys)
        for u, v in zip(x.keys + x.aggs, y.keys + y.aggs):
            np.testing.assert_array_equal(u, v)

    abc = [a, b, c]
    neg = [dataclasses_replace(p, neg=True) for p in abc]
    # NOT (a OR b) = NOT a AND NOT b
    same(q(abc, [P, A, ("or", 2), Cn]), q(neg[:2]))
    # NOT (a AND b) = NOT a OR NOT b
    same(q(abc, [P, A, ("and", 2), Cn]), q([dataclasses_replace(p, group=4) for p in neg[:2]]))
    # a AND (b OR c) = (a AND b) OR (a AND c)
    same(q(abc, [P, A, B, ("or", 2), ("and", 2)]), q(abc, [P, A, ("and", 2), P, B, ("and", 2), ("or", 2)]))
    # a OR (b AND c) = (a OR b) AND (a OR c), the second in OR-group form
    same(q(abc, [P, A, B, ("and", 2), ("or", 2)]),
         q([dataclasses_replace(a, group=1), dataclasses_replace(b, group=1),
            dataclasses_replace(a, group=2), dataclasses_replace(c, group=2)]))
    # NOT NOT a = a; a one-operand AND / OR is its operand
    same(q(abc, [P, Cn, Cn]), q([a]))
    same(q(abc, [P, ("and", 1), ("or", 1)]), q([a]))


# ---------------------------------------------------------------- random filters
@pytest.mark.parametrize("seed", range(40))
def test_random_trees_keep_the_set_algebra_rows(oracle_mod, seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(1, 120))
    k = int(rng.integers(1, 5))
    t, preds = _random_atoms(rng, n, k)
    prog = random_tree(rng, k, max_depth=int(rng.integers(1, 4)))
    want = set_algebra(prog, [pred_rows(t, p) for p in preds], n)
    assert kept_rows(oracle_mod, t, preds, prog) == sorted(want)


@pytest.mark.parametrize("seed", range(30))
def test_random_or_groups_keep_the_set_algebra_rows(oracle_mod, seed):
    """OR-group form: the AND of group-0 predicates and of each group's OR,
    with negated predicates complemented first."""
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(1, 120))
    t, preds = _random_atoms(rng, n, int(rng.integers(1, 6)))
    preds = random_or_groups(rng, preds)
    universe = set(range(n))
    want = set(universe)
    groups = {}
    for p in preds:
        r = pred_rows(t, dg.Pred(p.col, p.op, p.lo, p.hi, p.ints, p.strs))
        r = universe - r if p.neg else r
        if p.group == 0:
            want &= r
        else:
            groups[p.group] = groups.get(p.group, set()) | r
    for r in groups.values():
        want &= r
    assert kept_rows(oracle_mod, t, preds) == sorted(want)


@pytest.mark.parametrize("seed", range(30))
def test_random_filters_match_tensor_formulation(oracle_mod, seed):
    """Whole queries (keys and every aggregate) with random filter programs
    or OR groups against the numpy formulation (Plain masks combined with
    &, |, ~)."""
    rng = np.random.default_rng(6000 + seed)
    n = int(rng.integers(1, 300))
    cols = [random_column(rng, n, str(rng.choice(["rle", "plain", "packed", "index", "dict"]))) for _ in range(4)]
    t = dg.Table(cols, n)
    plan = random_plan(rng, t, n_preds=int(rng.integers(1, 5)))
    if seed % 2:
        plan = dg.Plan(plan.preds, plan.group_by, plan.aggs, filter=random_tree(rng, len(plan.preds)))
    else:
        plan = dg.Plan(random_or_groups(rng, plan.preds), plan.group_by, plan.aggs)
    assert_same(oracle_mod.query(t, plan), tensor_ref.query(t, plan))
    assert_same(oracle_mod.query(t, plan, n_threads=3, row_ranges=[(0, n // 2), (n // 2, n)]),
                tensor_ref.query(t, plan))


def test_every_filter_over_two_predicates_on_tiny_tables(oracle_mod):
    """Brute force: every table of N <= 4 rows with A in {0,1,2}^N (RLE) and
    every filter program of one OR / AND over the four literals a, NOT a,
    b, NOT b (a: A >= 1, b: A != 2)."""
    lits = [[("pred", 0)], [("pred", 0), ("not", 0)], [("pred", 1)], [("pred", 1), ("not", 0)]]
    preds = [dg.Pred(0, "ge", 1), dg.Pred(0, "ne", 2)]
    for n in range(1, 5):
        for av in itertools.product([0, 1, 2], repeat=n):
            v, e = dg.rle_encode(np.array(av, dtype=np.int64), np.int64)
            t = dg.Table([dg.RLE(v, e, n)], n)
            truth = [[x >= 1 for x in av], [x != 2 for x in av]]
            for l1, l2 in itertools.product(range(4), repeat=2):
                for op in ("and", "or"):
                    prog = lits[l1] + lits[l2] + [(op, 2)]

                    def lit(li, r):
                        x = truth[li // 2][r]
                        return not x if li % 2 else x

                    want = [r for r in range(n) if (lit(l1, r) and lit(l2, r) if op == "and" else lit(l1, r) or lit(l2, r))]
                    assert kept_rows(oracle_mod, t, preds, prog) == want


@pytest.mark.parametrize("prog,groups", [
    ([("and", 2)], False),                          # operands missing
    ([("not", 0)], False),
    ([("pred", 0), ("pred", 0)], False),            # two values left
    ([("pred", 3)], False),                         # no such predicate
    ([("pred", 0), ("or", 0)], False),              # zero operands
    ([("pred", 0), ("pred", 1), ("or", 3)], False),
    ([("pred", 0)], True),                          # OR groups with a program
])
def test_malformed_filters_are_rejected(oracle_mod, prog, groups):
    n = 10
    t = dg.Table([as_plain(np.arange(n))], n)
    preds = [dg.Pred(0, "lt", 5, group=2 if groups else 0), dg.Pred(0, "gt", 7)]
    with pytest.raises(ValueError):
        oracle_mod.query(t, dg.Plan(preds, [], [COUNT], filter=prog))
