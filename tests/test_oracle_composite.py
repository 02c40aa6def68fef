"""Pins of the oracle's composite encodings (Section 3.2 Composite
Encodings).  RLE + Index (runs for the pure stretches, Index for the
scattered rows, the two disjoint): the paper's [A,A,A,A,B,C,D] example,
decoding against the plain sequence, queries on the composite against the
same queries on the plain column, the rejection of gaps and overlaps.
Plain + Index (a narrow packed part, outliers listed): the paper's
[1, 2, 3, 10^10, 10^10] example with garbage in the ignored packed slots,
random columns with outliers decoded and queried against the plain column,
unsorted positions rejected."""
import json
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests import tensor_ref
from tests.test_oracle import assert_same
from tests.helpers import random_plan

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def letters(xs):
    return [ord(x) for x in xs]


def test_paper_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "rle_index_example.json")))
    seq = letters(g["sequence"])
    col = dg.RLEIndex(np.array(letters(g["rle"]["v"]), np.int64), np.array(g["rle"]["s"], np.int64),
                      np.array(g["rle"]["e"], np.int64) + 1,           # inclusive -> exclusive ends
                      np.array(letters(g["index"]["v"]), np.int64), np.array(g["index"]["p"], np.int64), len(seq))
    assert oracle_mod.decode(col).tolist() == seq
    # the encoder splits the sequence the paper's way (runs of at least 2)
    enc = dg.rle_index_encode(np.array(seq), 2)
    assert enc.run_values.tolist() == col.run_values.tolist()
    assert enc.run_starts.tolist() == col.run_starts.tolist() and enc.run_ends.tolist() == col.run_ends.tolist()
    assert enc.values.tolist() == col.values.tolist() and enc.positions.tolist() == col.positions.tolist()


def random_sequence(rng, n):
    """Long pure runs mixed with stretches of scattered values."""
    out, r = [], 0
    while r < n:
        if rng.random() < 0.5:
            L = int(rng.integers(1, 60))
            out += [int(rng.integers(-30, 30))] * L
        else:
            L = int(rng.integers(1, 20))
            out += rng.integers(-30, 30, size=L).tolist()
        r += L
    return np.array(out[:n], dtype=np.int64)


@pytest.mark.parametrize("seed", range(16))
def test_queries_match_the_plain_column(oracle_mod, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 3000))
    seqs = [random_sequence(rng, n) for _ in range(3)]
    mins = [int(rng.integers(1, 8)) for _ in range(3)]
    comp = dg.Table([dg.rle_index_encode(s, m) for s, m in zip(seqs, mins)], n)
    plain = dg.Table([dg.Plain(s) for s in seqs], n)
    for c, s in zip(comp.columns, seqs):
        assert oracle_mod.decode(c).tolist() == s.tolist()
    plan = random_plan(rng, plain)
    a, b = oracle_mod.query(comp, plan), oracle_mod.query(plain, plan)
    assert [x.tolist() for x in a.keys] == [x.tolist() for x in b.keys]
    assert [x.tolist() for x in a.aggs] == [x.tolist() for x in b.aggs]
    assert_same(a, tensor_ref.query(comp, plan))


def test_gaps_and_overlaps_are_rejected(oracle_mod):
    ok = dg.RLEIndex(np.array([1, 2]), np.array([0, 5]), np.array([3, 8]), np.array([7, 9]), np.array([3, 4]), 8)
    oracle_mod.decode(ok)
    t = dg.Table([ok], 8)
    oracle_mod.query(t, dg.Plan([], [], [dg.Agg("sum", 0)]))
    bad = [
        dg.RLEIndex(np.array([1, 2]), np.array([0, 5]), np.array([3, 8]), np.array([7]), np.array([3]), 8),   # gap at 4
        dg.RLEIndex(np.array([1, 2]), np.array([0, 4]), np.array([5, 8]), np.array([7]), np.array([4]), 8),   # overlap
        dg.RLEIndex(np.array([1, 2]), np.array([5, 0]), np.array([8, 3]), np.array([7, 9]), np.array([3, 4]), 8),
        dg.RLEIndex(np.array([1, 2]), np.array([0, 5]), np.array([3, 8]), np.array([7, 9]), np.array([3, 4]), 9),
    ]
    for c in bad:
        with pytest.raises(ValueError, match="status -1"):
            oracle_mod.query(dg.Table([c], c.n_rows), dg.Plan([], [], [dg.Agg("sum", 0)]))


# ---------------------------------------------------------------- Plain + Index
def test_plain_index_paper_example(oracle_mod):
    """[1, 2, 3, 10^10, 10^10]: the regular values in a narrow packed part,
    the outliers at 3 and 4 listed; the packed fields at the listed rows hold
    garbage that decoding never reads."""
    g = json.load(open(os.path.join(GOLDEN, "plain_index_example.json")))
    n = len(g["column"])
    fields = np.array(g["plain"] + [7, 5], dtype=np.uint64)        # 7, 5: the ignored slots
    col = dg.PackedIndex(dg.pack_bits(fields, 3), 3, 0, np.array(g["index"]["v"], np.int64),
                         np.array(g["index"]["p"], np.int64), n)
    assert oracle_mod.decode(col).tolist() == g["column"]
    enc = dg.packed_index_encode(np.array(g["column"]), 3)
    assert enc.positions.tolist() == g["index"]["p"] and enc.values.tolist() == g["index"]["v"]
    assert oracle_mod.decode(enc).tolist() == g["column"]


@pytest.mark.parametrize("seed", range(12))
def test_plain_index_queries_match_the_plain_column(oracle_mod, seed):
    rng = np.random.default_rng(950 + seed)
    n = int(rng.integers(1, 3000))
    seqs = []
    for _ in range(3):
        v = rng.integers(-100, 100, size=n).astype(np.int64)
        out = rng.random(n) < float(rng.choice([0.0, 0.01, 0.2]))
        v[out] = rng.integers(-(1 << 40), 1 << 40, size=int(out.sum()))
        seqs.append(v)
    w = int(rng.integers(8, 12))
    comp = dg.Table([dg.packed_index_encode(s, w, fill=rng.integers(0, 1 << w, size=n)) for s in seqs], n)
    plain = dg.Table([dg.Plain(s) for s in seqs], n)
    for c, s in zip(comp.columns, seqs):
        assert oracle_mod.decode(c).tolist() == s.tolist()
    plan = random_plan(rng, plain)
    a, b = oracle_mod.query(comp, plan), oracle_mod.query(plain, plan)
    assert [x.tolist() for x in a.keys] == [x.tolist() for x in b.keys]
    assert [x.tolist() for x in a.aggs] == [x.tolist() for x in b.aggs]
    assert_same(a, tensor_ref.query(comp, plan))


def test_plain_index_unsorted_positions_are_rejected(oracle_mod):
    col = dg.PackedIndex(dg.pack_bits(np.zeros(5, np.uint64), 2), 2, 0, np.array([9, 8]), np.array([3, 1]), 5)
    with pytest.raises(ValueError, match="status -1"):
        oracle_mod.query(dg.Table([col], 5), dg.Plan([], [], [dg.Agg("sum", 0)]))
