"""The synthetic workloads follow their stated recipes (shapes, sizes, value
ranges and distributions), so that the benchmarked inputs are what the
documentation says they are."""
import numpy as np

from paper_2506_10092_gb300 import datagen as dg


def _run_lengths(c):
    return np.diff(np.concatenate([[0], c.run_ends.astype(np.int64)]))


def test_tiny_two_rle_recipe():
    t, plan = dg.tiny_two_rle(1_000_000, seed=3)
    a, b = t.columns
    assert a.run_ends.dtype == np.int32 and int(a.run_ends[-1]) == 1_000_000
    assert 7.5 < _run_lengths(a).mean() < 8.5 and 4.7 < _run_lengths(b).mean() < 5.3
    assert a.run_values.min() >= 0 and a.run_values.max() == 99
    assert b.run_values.min() == 0 and b.run_values.max() == 9
    assert plan.preds[0].op == "lt" and plan.preds[0].lo == 50 and plan.group_by == [1]


def test_heterogeneous_recipe():
    n = 400_000
    t, plan = dg.heterogeneous(n, seed=4)
    c1, c2, c3, c4, c5 = t.columns
    assert 800 < _run_lengths(c1).mean() < 1200 and c1.run_values.max() <= 999   # ~400 runs sampled
    assert len(c2.strings) == 10_000 and c2.bit_width == 14
    assert all(8 <= len(s) <= 24 for s in c2.strings) and c2.strings == sorted(c2.strings)
    assert c3.positions.shape[0] == n // 100 and c3.default == 0
    assert np.all(np.diff(c3.positions) > 0) and np.abs(c3.values).max() <= 1 << 40
    assert c4.values.dtype == np.int32 and c4.values.min() >= 0 and c4.values.max() <= 1_000_000
    assert c5.bit_width == 20 and c5.base == (1 << 32) + 12345
    # Zipf(1.1) over 10,000 ranks: the most frequent code holds ~1/H(10000, 1.1) of the rows
    from oracle import oracle
    codes = oracle.decode(c2)
    top = np.bincount(codes, minlength=10_000).max() / n
    h = (np.arange(1, 10_001, dtype=np.float64) ** -1.1).sum()
    assert abs(top - 1 / h) < 0.02
    assert len(plan.preds[0].strs) == 64 and plan.preds[1].lo == 250_000 and plan.preds[1].hi == 749_999


def test_partition_sizes_are_log_uniform():
    rng = np.random.default_rng(1)
    s = dg.partition_sizes(rng, 20_000)
    logs = np.log(s)
    lo, hi = np.log(1e4), np.log(5e7)
    # uniform in log space: mean and quartiles of the logs
    assert abs(logs.mean() - (lo + hi) / 2) < 0.05
    q1, q3 = np.percentile(logs, [25, 75])
    assert abs(q1 - (lo + (hi - lo) / 4)) < 0.1 and abs(q3 - (lo + 3 * (hi - lo) / 4)) < 0.1


def test_batch_query_literals():
    rng = np.random.default_rng(2)
    qs = dg.batch_queries(rng, 2000, 16)
    thresholds = [p.preds[0].lo for _, k, p in qs if k == "tiny"]
    assert min(thresholds) >= 0 and max(thresholds) <= 99
    for _, k, p in qs:
        if k == "nested":
            assert 0 <= p.preds[0].lo <= p.preds[0].hi <= 999
            assert p.group_by == [1, 3] and [a.col for a in p.aggs] == [4, 5]
