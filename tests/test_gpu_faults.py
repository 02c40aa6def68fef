"""Failure paths on the GPU without faulting it: a device wait that nothing
completes ends by itself with CQ_ERR_TIMEOUT and the context stays usable;
device-detected data errors come back as statuses with their detail."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_survives(oracle_mod):
    from paper_2506_10092_gb300 import cq
    ctx = cq.cq_ctx_create(0)
    for limit_us in (1000, 20000):
        assert cq.cq_selftest_bounded_wait(ctx, limit_us) == cq.CQ_ERR_TIMEOUT
    table, plan = dg.tiny_two_rle(100_000, seed=9)
    t, cols = cq.table_from(ctx, table)
    got = cq.fetch_all(cq.cq_query_run(t, plan))
    ref = oracle_mod.query(table, plan)
    for g, w in zip(got, ref.keys + ref.aggs):
        np.testing.assert_array_equal(g, w)


def test_self_test_rejects_bad_limits():
    from paper_2506_10092_gb300 import cq
    ctx = cq.cq_ctx_create(0)
    for bad in (0, 10_000_000):
        with pytest.raises(cq.CQError) as e:
            cq.cq_selftest_bounded_wait(ctx, bad)
        assert e.value.status == cq.CQ_ERR_INVALID_ARG
