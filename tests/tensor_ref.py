"""The paper's own tensor formulation of a filter / group-by / aggregate query,
written with numpy library primitives, used only to pin the C++ oracle.

It follows the PyTorch program of the paper rather than the oracle's row
loop: RLE columns are expanded with ``repeat`` (``repeat_interleave``,
Section 2.2), Index columns by indexed assignment, grouping uses ``unique``
with inverse indices and aggregation uses scatter-style ``ufunc.at``
(Section 7, grouping and aggregating phases).  Sums are exact Python ints.
Bit-packed fields are read from a Python big-int bit stream, which is the
definition of an LSB-first stream.  Small inputs only.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def decode_bits(words: np.ndarray, w: int, n: int) -> np.ndarray:
    stream = 0
    for k, x in enumerate(np.asarray(words, dtype=np.uint64).tolist()):
        stream |= int(x) << (32 * k)
    mask = (1 << w) - 1
    return np.array([(stream >> (i * w)) & mask for i in range(n)], dtype=object)


def decode(col) -> np.ndarray:
    """Python-int object array of the column's logical values (DICT: codes)."""
    if col.enc == "rle":
        ends = np.asarray(col.run_ends, dtype=np.int64)
        lens = np.diff(np.concatenate([[0], ends]))
        return np.repeat(np.asarray(col.run_values, dtype=np.int64), lens).astype(object)
    if col.enc == "index":
        out = np.full(col.n_rows, int(col.default), dtype=object)
        out[np.asarray(col.positions, dtype=np.int64)] = [int(v) for v in np.asarray(col.values)]
        return out
    if col.enc == "packed":
        return decode_bits(col.words, col.bit_width, col.n_rows) + int(col.base)
    if col.enc == "dict":
        return decode_bits(col.words, col.bit_width, col.n_rows)
    if col.enc == "plain":
        return np.asarray(col.values, dtype=np.int64).astype(object)
    if col.enc == "packed_index":
        out = decode_bits(col.words, col.bit_width, col.n_rows) + int(col.base)
        for v, p in zip(np.asarray(col.values).tolist(), np.asarray(col.positions).tolist()):
            out[p] = int(v)
        return out
    if col.enc == "rle_index":
        out = np.empty(col.n_rows, dtype=object)
        for v, s, e in zip(np.asarray(col.run_values).tolist(), np.asarray(col.run_starts).tolist(),
                           np.asarray(col.run_ends).tolist()):
            out[s:e] = int(v)
        for v, p in zip(np.asarray(col.values).tolist(), np.asarray(col.positions).tolist()):
            out[p] = int(v)
        return out
    raise ValueError(col.enc)


def _pred_mask(col, vals, p) -> np.ndarray:
    if col.enc == "dict":
        strings = col.strings
        lits = [bytes(x) for x in (p.strs or [])]

        def f(code):
            s = strings[int(code)]
            if p.op == "in":
                return s in lits
            a = lits[0]
            return {"lt": s < a, "le": s <= a, "gt": s > a, "ge": s >= a, "eq": s == a, "ne": s != a,
                    "between": lits[0] <= s <= lits[-1] if len(lits) > 1 else False}[p.op]
        return np.array([f(v) for v in vals], dtype=bool)
    if p.op == "in":
        allowed = set(int(x) for x in p.ints)
        return np.array([int(v) in allowed for v in vals], dtype=bool)
    lo, hi = int(p.lo), int(p.hi)
    ops = {"lt": lambda v: v < lo, "le": lambda v: v <= lo, "gt": lambda v: v > lo, "ge": lambda v: v >= lo,
           "eq": lambda v: v == lo, "ne": lambda v: v != lo, "between": lambda v: lo <= v <= hi}
    return np.array([ops[p.op](int(v)) for v in vals], dtype=bool)


def filter_mask(plan, masks, n) -> np.ndarray:
    """Combine Plain masks with the logical operators of Section 5 (``&``,
    ``|``, ``~``): each predicate's mask is complemented when negated; a
    filter program is run on a stack of masks, else the masks of or_group 0
    and the OR of each group's masks are AND-ed."""
    masks = [~m if getattr(p, "neg", False) else m for p, m in zip(plan.preds, masks)]
    prog = getattr(plan, "filter", None)
    if prog:
        st = []
        for kind, arg in prog:
            if kind == "pred":
                st.append(masks[arg])
            elif kind == "not":
                st.append(~st.pop())
            else:
                top = [st.pop() for _ in range(arg)]
                acc = top[0]
                for m in top[1:]:
                    acc = (acc & m) if kind == "and" else (acc | m)
                st.append(acc)
        assert len(st) == 1
        return st[0]
    out = np.ones(n, dtype=bool)
    groups = {}
    for p, m in zip(plan.preds, masks):
        g = getattr(p, "group", 0)
        if g == 0:
            out &= m
        else:
            groups[g] = groups[g] | m if g in groups else m
    for m in groups.values():
        out &= m
    return out


def query(table, plan):
    """Returns (keys: list of int arrays, aggs: list of arrays, overflow: bool)."""
    n = table.n_rows
    flat = {}
    for i in set([p.col for p in plan.preds] + list(plan.group_by) + [a.col for a in plan.aggs if a.op != "count"]
                 + [a.col2 for a in plan.aggs if getattr(a, "expr", None)]):
        flat[i] = decode(table.columns[i])
    mask = filter_mask(plan, [_pred_mask(table.columns[p.col], flat[p.col], p) for p in plan.preds], n)
    rows = np.flatnonzero(mask)
    if plan.group_by:
        if len(rows):
            # unique with inverse indices (torch.unique); tuples of exact ints
            tuples = [tuple(int(flat[c][r]) for c in plan.group_by) for r in rows]
            uniq = sorted(set(tuples))
            pos = {t: i for i, t in enumerate(uniq)}
            inv = np.array([pos[t] for t in tuples], dtype=np.int64)
        else:
            uniq, inv = [], np.zeros(0, dtype=np.int64)
        G = len(uniq)
    else:
        uniq, inv, G = [()], np.zeros(len(rows), dtype=np.int64), 1
    count = np.bincount(inv, minlength=G).astype(np.uint64)
    aggs = []
    overflow = False
    for a in plan.aggs:
        if a.op == "count":
            aggs.append(count)
            continue
        v = flat[a.col][rows]
        if getattr(a, "expr", None):
            # position-wise arithmetic on the (aligned) rows, exact Python ints
            w = flat[a.col2][rows]
            f = {"add": lambda x, y: x + y, "sub": lambda x, y: x - y, "mul": lambda x, y: x * y}[a.expr]
            v = np.array([f(int(x), int(y)) for x, y in zip(v.tolist(), w.tolist())], dtype=object)
            if any(x > 2**63 - 1 or x < -2**63 for x in v.tolist()):
                raise ValueError("expression value outside int64")
        col = table.columns[a.col]
        if a.op in ("var_pop", "var_samp", "std_pop", "std_samp"):
            # Section 7: from COUNT, SUM and the sum of squares; the exact
            # rational rounded once (Fraction -> float), STD its square root
            s1, s2, cnt = [0] * G, [0] * G, [0] * G
            for g, x in zip(inv.tolist(), v.tolist()):
                s1[g] += int(x)
                s2[g] += int(x) * int(x)
                cnt[g] += 1
            out = []
            for g in range(G):
                n_, d = cnt[g], cnt[g] - (1 if a.op.endswith("samp") else 0)
                var = float(Fraction(n_ * s2[g] - s1[g] * s1[g], n_ * d)) if n_ and d else 0.0
                out.append(math.sqrt(var) if a.op.startswith("std") else var)
            aggs.append(np.array(out, dtype=np.float64))
            continue
        if a.op in ("sum", "avg"):
            s = [0] * G
            for g, x in zip(inv.tolist(), v.tolist()):        # scatter(reduce=sum)
                s[g] += int(x)
            if a.op == "sum":
                if any(x > 2**63 - 1 or x < -2**63 for x in s):
                    overflow = True
                aggs.append(np.array([x if -2**63 <= x < 2**63 else 0 for x in s], dtype=np.int64))
            else:
                aggs.append(np.array([float(s[g]) / float(int(count[g])) if count[g] else 0.0 for g in range(G)]))
        else:
            best = [None] * G
            for g, x in zip(inv.tolist(), v.tolist()):
                x = int(x)
                if col.enc == "dict":
                    k = col.strings[x]
                    if best[g] is None or (k < col.strings[best[g]] if a.op == "min" else k > col.strings[best[g]]):
                        best[g] = x
                elif best[g] is None or (x < best[g] if a.op == "min" else x > best[g]):
                    best[g] = x
            aggs.append(np.array([0 if b is None else b for b in best], dtype=np.int64))
    keys_out = [np.array([u[k] for u in uniq], dtype=np.int64) for k in range(len(plan.group_by))]
    return keys_out, aggs, overflow
