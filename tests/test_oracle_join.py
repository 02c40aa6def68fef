"""Pins of the oracle's join primitives (the paper's Join Operations
section: Get Join Index, then Apply Join Index).  The pins: the paper's
R.A = S.B example (its printed index tensors and result column), the
appendix's Plain x RLE example (its index tensors, as a multiset of row
pairs), brute force against nested loops, the count as the sum over values
of the product of their multiplicities, and RLE x RLE counts as products of
run lengths."""
import json
import os
from collections import Counter

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, rle_inclusive

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load():
    return json.load(open(os.path.join(GOLDEN, "join_examples.json")))


def codes(xs):
    return np.array([ord(x) for x in xs], dtype=np.int64)


def test_paper_example(oracle_mod):
    g = load()["rs_example"]
    ra, sb, sc = dg.Plain(codes(g["R_A"])), dg.Plain(codes(g["S_B"])), dg.Plain(codes(g["S_C"]))
    li, ri = oracle_mod.join_index(ra, sb)
    assert li.tolist() == g["left_index"] and ri.tolist() == g["right_index"]
    assert oracle_mod.apply_join_index(sc, ri).tolist() == codes(g["result"]).tolist()


def test_plain_rle_example(oracle_mod):
    g = load()["plain_rle_example"]
    plain = dg.Plain(codes(g["plain"]))
    rle = rle_inclusive(codes(g["rle"]["v"]), g["rle"]["s"], g["rle"]["e"])
    li, ri = oracle_mod.join_index(plain, rle)
    # the paper's tensors: the RLE join index (v = run index, s..e = rows)
    # expanded to rows lines up entry by entry with the Plain join index
    ji = g["rle_index"]
    rows = [r for s, e in zip(ji["s"], ji["e"]) for r in range(s, e + 1)]
    assert len(rows) == len(g["plain_index"])
    want = Counter(zip(g["plain_index"], rows))
    assert Counter(zip(li.tolist(), ri.tolist())) == want
    # each run index in the RLE join index names the run holding those rows
    for v, s, e in zip(ji["v"], ji["s"], ji["e"]):
        assert g["rle"]["s"][v] <= s and e <= g["rle"]["e"][v]


@pytest.mark.parametrize("seed", range(20))
def test_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(1200 + seed)
    encs = ["rle", "plain", "packed", "index"]
    a = random_column(rng, int(rng.integers(0, 300)), str(rng.choice(encs)), lo=-6, hi=6)
    b = random_column(rng, int(rng.integers(0, 300)), str(rng.choice(encs)), lo=-6, hi=6)
    va, vb = oracle_mod.decode(a), oracle_mod.decode(b)
    li, ri = oracle_mod.join_index(a, b)
    want = [(i, j) for i in range(len(va)) for j in range(len(vb)) if va[i] == vb[j]]
    assert list(zip(li.tolist(), ri.tolist())) == want
    ca, cb = Counter(va.tolist()), Counter(vb.tolist())
    assert len(li) == sum(ca[v] * cb[v] for v in ca)
    assert oracle_mod.apply_join_index(b, ri).tolist() == oracle_mod.apply_join_index(a, li).tolist()


def test_rle_by_rle_counts_are_products_of_run_lengths(oracle_mod):
    rng = np.random.default_rng(3)
    n = 5000
    a = dg.make_rle(rng, n, 40.0, 0, 9, np.int64, np.int64)
    b = dg.make_rle(rng, n, 25.0, 0, 9, np.int64, np.int64)
    li, _ = oracle_mod.join_index(a, b)
    la = np.diff(np.concatenate([[0], a.run_ends]))
    lb = np.diff(np.concatenate([[0], b.run_ends]))
    want = sum(int(x) * int(y) for va, x in zip(a.run_values, la) for vb, y in zip(b.run_values, lb) if va == vb)
    assert len(li) == want


def test_rows_out_of_range_are_rejected(oracle_mod):
    with pytest.raises(ValueError, match="status -1"):
        oracle_mod.apply_join_index(dg.Plain(np.arange(3, dtype=np.int64)), [0, 3])
