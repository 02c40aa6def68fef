"""Small table builders shared by the tests (no query arithmetic here)."""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2506_10092_gb300 import datagen as dg


def rle_inclusive(vals, starts, ends, n_rows=None, val_dtype=np.int64, end_dtype=np.int64):
    """RLE column from the paper's inclusive (start, end) form; the runs must
    cover 0..n_rows-1 without gaps."""
    starts = np.asarray(starts, dtype=np.int64)
    ends = np.asarray(ends, dtype=np.int64)
    assert starts[0] == 0 and np.all(starts[1:] == ends[:-1] + 1)
    n = int(ends[-1] + 1) if n_rows is None else int(n_rows)
    return dg.RLE(np.asarray(vals, dtype=val_dtype), (ends + 1).astype(end_dtype), n)


def mask_rle(ranges, n_rows):
    """RLE 0/1 column that is 1 on the inclusive ranges [(s, e), ...] and 0 elsewhere."""
    plain = np.zeros(n_rows, dtype=np.int64)
    for s, e in ranges:
        plain[s:e + 1] = 1
    v, e = dg.rle_encode(plain, np.int64)
    return dg.RLE(v, e, n_rows)


def as_plain(values):
    return dg.Plain(np.asarray(values, dtype=np.int64))


def random_column(rng, n, enc, lo=-50, hi=50, dict_strings=None):
    """A column of the requested encoding with values in lo..hi."""
    if enc == "rle":
        ends = dg.geometric_ends(rng, n, float(rng.choice([1.5, 3.0, 10.0])), np.int64)
        vals = rng.integers(lo, hi + 1, size=ends.shape[0])
        return dg.RLE(vals.astype(np.int64), ends, n)
    if enc == "plain":
        return dg.Plain(rng.integers(lo, hi + 1, size=n).astype(np.int64))
    if enc == "packed":
        w = int(rng.integers(1, 12))
        base = int(rng.integers(lo, hi + 1))
        return dg.make_packed(rng.integers(0, 1 << w, size=n).astype(np.uint64), w, base)
    if enc == "index":
        nnz = int(rng.integers(0, n + 1))
        pos = np.sort(rng.choice(n, size=nnz, replace=False)).astype(np.int64)
        return dg.Index(rng.integers(lo, hi + 1, size=nnz).astype(np.int64), pos, int(rng.integers(lo, hi + 1)), n)
    if enc == "dict":
        strings = dict_strings or dg.random_strings(rng, int(rng.integers(1, 20)), 1, 4)
        w = max(1, int(np.ceil(np.log2(max(2, len(strings))))))
        codes = rng.integers(0, len(strings), size=n).astype(np.uint64)
        return dg.make_dict(strings, codes, w)
    raise ValueError(enc)


def random_plan(rng, table, n_preds=None, n_gb=None, allow=("sum", "count", "min", "max", "avg")):
    ncol = len(table.columns)
    preds = []
    for _ in range(int(rng.integers(0, 3)) if n_preds is None else n_preds):
        c = int(rng.integers(0, ncol))
        col = table.columns[c]
        if col.enc == "dict":
            op = str(rng.choice(["in", "lt", "ge", "eq", "between"]))
            picks = [col.strings[int(i)] for i in rng.integers(0, len(col.strings), size=3)]
            picks.append(b"zz-not-in-dict")
            if op == "between":
                a, b = sorted(picks[:2])
                preds.append(dg.Pred(c, op, strs=[a, b]))
            elif op == "in":
                preds.append(dg.Pred(c, op, strs=picks))
            else:
                preds.append(dg.Pred(c, op, strs=[picks[0]]))
        else:
            op = str(rng.choice(["lt", "le", "gt", "ge", "eq", "ne", "between", "in"]))
            lo, hi = sorted(int(x) for x in rng.integers(-60, 60, size=2))
            if op == "in":
                preds.append(dg.Pred(c, op, ints=[int(x) for x in rng.integers(-60, 60, size=5)]))
            else:
                preds.append(dg.Pred(c, op, lo, hi))
    k = int(rng.integers(0, 3)) if n_gb is None else n_gb
    gb = [int(x) for x in rng.choice(ncol, size=min(k, ncol), replace=False)]
    aggs = [dg.Agg("count")]
    for _ in range(int(rng.integers(1, 4))):
        c = int(rng.integers(0, ncol))
        ops = [o for o in allow if o != "count"]
        if table.columns[c].enc == "dict":
            ops = [o for o in ops if o in ("min", "max")] or ["count"]
        aggs.append(dg.Agg(str(rng.choice(ops)), c))
    return dg.Plan(preds, gb, aggs)


def random_tree(rng, n_preds, max_depth=3):
    """A random boolean expression over predicates 0..n_preds-1 as a postfix
    program of ("pred", i), ("not", 0), ("and", k), ("or", k) nodes."""
    out = []

    def build(d):
        r = rng.random()
        if d == 0 or r < 0.3:
            out.append(("pred", int(rng.integers(0, n_preds))))
            if rng.random() < 0.3:
                out.append(("not", 0))
        elif r < 0.4:
            build(d - 1)
            out.append(("not", 0))
        else:
            k = int(rng.integers(1, 4))
            for _ in range(k):
                build(d - 1)
            out.append((str(rng.choice(["and", "or"])), k))

    build(max_depth)
    return out


def random_or_groups(rng, preds):
    """The predicates with random OR groups (0 = a conjunct of its own) and
    random negation."""
    out = []
    for p in preds:
        g = int(rng.integers(0, 3))
        out.append(dataclasses.replace(p, group=g, neg=bool(rng.random() < 0.35)))
    return out

