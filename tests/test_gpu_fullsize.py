"""Parity at the benchmarked sizes, in the launch configurations bench.py
times: the heterogeneous 100M-row query in full, the 20-billion-row nested
table on sampled groups, and the batched workload's full partition pool on
sampled queries.  The oracle computes each sampled output exactly from the
rows that feed it."""
import os

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

SEED = dg.DEFAULT_SEED


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


@pytest.fixture(scope="module")
def ctx(cq):
    return cq.cq_ctx_create(0)


def check(got, ref, msg):
    want = ref.keys + ref.aggs
    assert len(got) == len(want), msg
    for i, (g, w) in enumerate(zip(got, want)):
        assert g.dtype == w.dtype, (msg, i)
        np.testing.assert_array_equal(g, w, err_msg=f"{msg} output column {i}")


def test_heterogeneous_100m_rows_in_full(cq, ctx, oracle_mod):
    table, plan = dg.heterogeneous(100_000_000, seed=SEED)
    t, cols = cq.table_from(ctx, table)
    got = cq.fetch_all(cq.cq_query_run(t, plan))
    check(got, oracle_mod.query(table, plan, n_threads=oracle_mod.cores()), "heterogeneous 100M")


def test_nested_20b_rows_sampled_groups(cq, ctx, oracle_mod):
    """GROUP BY c2, c4 over 20e9 rows: every group of a sampled c2 value is
    recomputed by the oracle from exactly the rows holding that value (the
    union of its c2 runs)."""
    from paper_2506_10092_gb300 import devgen
    n = 20_000_000_000
    dn = devgen.DeviceNested(cq, ctx, n, seed=SEED)
    plan = dg.nested_plan(lean=True)
    k2, k4, s7, s8 = cq.fetch_all(cq.cq_query_run(dn.table, plan))
    assert len(k2) > 100_000
    assert np.all(np.diff(k2) >= 0)                      # key order
    c2 = dn.runs[1]
    rng = np.random.default_rng(7)
    values = [int(c2.run_values.min()), int(c2.run_values.max())] + \
        [int(v) for v in rng.choice(np.unique(c2.run_values), size=3, replace=False)]
    cores = oracle_mod.cores()
    for v in values:
        sub = dg.nested_subtable(dn.runs, SEED, dg.value_ranges(c2, v))
        ref = oracle_mod.query(sub, plan, n_threads=cores)
        m = k2 == v
        check([k2[m], k4[m], s7[m], s8[m]], ref, f"c2 = {v}")


def test_batched_full_pool_sampled_queries(cq, ctx, oracle_mod):
    """The batched workload as bench.py builds it (256 partitions, 4096
    queries, autotuned shape); sampled queries against the oracle on their
    own partitions."""
    import argparse
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import torch
    args = argparse.Namespace(seed=SEED, parts=256, part_max=5e7)
    sizes, parts = bench.build_pool(args, cq, ctx, torch)
    rng = np.random.default_rng([SEED, 5])
    qs = dg.batch_queries(rng, 4096, len(parts), lean=True)
    handles = [parts[p]["tiny"][1] if k == "tiny" else parts[p]["nested"].table for p, k, _ in qs]
    plans = [cq.PlanStruct(pl) for _, _, pl in qs]
    cq.cq_batch_tune(handles, plans)
    res = cq.cq_batch_run(handles, plans)
    # every kind of partition size: the smallest ones, and a few large ones
    order = np.argsort([parts[p]["n"] for p, _, _ in qs])
    sample = list(order[:12]) + list(order[len(order) // 2:len(order) // 2 + 3]) + list(order[-2:])
    for i in sample:
        p, kind, plan = qs[i]
        host = parts[p]["tiny"][0] if kind == "tiny" else parts[p]["nested"].host_table()
        ref = oracle_mod.query(host, plan, n_threads=oracle_mod.cores())
        check(cq.fetch_all(res[i]), ref, f"query {i} ({kind}, {parts[p]['n']} rows)")
