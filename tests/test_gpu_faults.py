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


_ALLOC_CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2506_10092_gb300 import cq, datagen as dg
from oracle import oracle
ctx = cq.cq_ctx_create(0)
table, plan = dg.tiny_two_rle(20000, seed=2)
fails, got = [], None
for _ in range(3):
    try:
        t, cols = cq.table_from(ctx, table)
        got = cq.fetch_all(cq.cq_query_run(t, plan))
        break
    except cq.CQError as e:
        fails.append(e.status)
ref = oracle.query(table, plan)
ok = got is not None and all((g == w).all() for g, w in zip(got, ref.keys + ref.aggs))
print(json.dumps({"fails": fails, "ok": bool(ok)}))
'''


@pytest.mark.parametrize("k", [1, 3, 6, 7])
def test_injected_allocation_failure_is_reported_and_recovered(k):
    """Host-side fault injection: the k-th device allocation of a process
    fails (column copies, validation scratch, the query's block).  The call
    that hit it returns CQ_ERR_OOM, nothing leaks into later calls, and the
    retry gives the oracle's result."""
    import json
    import os
    import subprocess
    import sys
    from paper_2506_10092_gb300 import cq
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CQ_FAULT_INJECT=f"alloc:{k}")
    out = subprocess.run([sys.executable, "-c", _ALLOC_CHILD, root], env=env, capture_output=True, text=True,
                         timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["ok"] and d["fails"] == [cq.CQ_ERR_OOM], d


_EVENT_CHILD = r'''
import json, sys, threading
sys.path.insert(0, sys.argv[1])
from paper_2506_10092_gb300 import cq, datagen as dg
from oracle import oracle
ctx = cq.cq_ctx_create(0)
table, plan = dg.tiny_two_rle(20000, seed=3)
t, cols = cq.table_from(ctx, table)
srv = cq.cq_server_create(ctx)
statuses = []
for _ in range(2):
    tk = cq.cq_server_submit(srv, t, plan)
    try:
        res, _lat = cq.cq_server_wait(srv, tk, timeout_us=30_000_000)
        got = cq.fetch_all(res)
        statuses.append(0)
    except cq.CQError as e:
        statuses.append(e.status)
ref = oracle.query(table, plan)
ok = all((g == w).all() for g, w in zip(got, ref.keys + ref.aggs))
done = threading.Event()
threading.Thread(target=lambda: (srv.close(), done.set()), daemon=True).start()
print(json.dumps({"statuses": statuses, "ok": bool(ok), "destroyed": done.wait(60)}))
'''


def test_serving_loop_fails_a_launch_whose_completion_reports_an_error():
    """Host-side fault injection (no GPU fault): the serving loop's first poll
    of a launch in flight reports a launch failure.  That query ends with
    CQ_ERR_CUDA instead of waiting forever, the next query gets the oracle's
    result, and the server shuts down."""
    import json
    import os
    import subprocess
    import sys
    from paper_2506_10092_gb300 import cq
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CQ_FAULT_INJECT="event:1")
    out = subprocess.run([sys.executable, "-c", _EVENT_CHILD, root], env=env, capture_output=True, text=True,
                         timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["statuses"] == [cq.CQ_ERR_CUDA, 0], d
    assert d["ok"] and d["destroyed"], d
