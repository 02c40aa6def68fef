"""The serving loop: queries submitted from several threads at random times
over resident tables, batched as they arrive.  Each result must equal the
query's result alone (cq_query_run) and the oracle's, bit for bit."""
import threading
import time

import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


@pytest.fixture(scope="module")
def ctx(cq):
    return cq.cq_ctx_create(0)


@pytest.fixture(scope="module")
def tables(cq, ctx):
    """One table per template: two-RLE, heterogeneous, nested."""
    out = {}
    tiny, _ = dg.tiny_two_rle(300_000, seed=41)
    het, het_plan = dg.heterogeneous(400_000, seed=42)
    nest, _ = dg.nested(700_000, seed=43, lean=True)
    for name, t in (("tiny", tiny), ("het", het), ("nest", nest)):
        out[name] = (t,) + tuple(cq.table_from(ctx, t))
    out["het_plan"] = het_plan
    return out


def mix(rng, tables, n):
    """Queries of the three templates, 60/30/10, with random literals."""
    qs = []
    for _ in range(n):
        u = rng.random()
        if u < 0.6:
            qs.append(("tiny", dg.tiny_plan(int(rng.integers(0, 100)))))
        elif u < 0.9:
            p = tables["het_plan"]
            lo = int(rng.integers(0, 900_000))
            qs.append(("het", dg.Plan([p.preds[0], dg.Pred(3, "between", lo, lo + 300_000)], p.group_by, p.aggs)))
        else:
            lo = int(rng.integers(0, 1000))
            qs.append(("nest", dg.nested_plan(lo, min(999, lo + int(rng.integers(0, 600))), lean=True)))
    return qs


def check(got, ref, msg):
    want = ref.keys + ref.aggs
    assert len(got) == len(want), msg
    for i, (g, w) in enumerate(zip(got, want)):
        assert g.dtype == w.dtype, (msg, i)
        np.testing.assert_array_equal(g, w, err_msg=f"{msg} output column {i}")


@pytest.mark.parametrize("n_streams,max_batch,budget,large_log2",
                         [(2, 256, 0, 0), (4, 8, 0, 18), (2, 32, 0, 16), (1, 64, 24 << 20, 0)])
def test_each_result_is_the_same_alone_and_in_the_mix(cq, ctx, tables, oracle_mod, n_streams, max_batch, budget,
                                                     large_log2):
    """Two lanes (large tables alone, small ones batched; large_log2 moves the
    heterogeneous and nested tables into the large lane) and one lane."""
    rng = np.random.default_rng(1000 + n_streams * 7 + max_batch)
    qs = mix(rng, tables, 120)
    srv = cq.cq_server_create(ctx, cq.server_options(memory_budget_bytes=budget, max_batch=max_batch,
                                                     n_streams=n_streams, max_wait_us=100,
                                                     large_rows_log2=large_log2))
    tickets = [None] * len(qs)
    delays = rng.exponential(200e-6, size=len(qs))          # Poisson arrivals, ~5000 q/s

    def submitter(idx):
        for i in idx:
            time.sleep(float(delays[i]))
            name, plan = qs[i]
            tickets[i] = cq.cq_server_submit(srv, tables[name][1], plan)

    order = rng.permutation(len(qs))
    threads = [threading.Thread(target=submitter, args=(order[k::3],)) for k in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in rng.permutation(len(qs)):                     # collected in random order
        res, lat = cq.cq_server_wait(srv, tickets[i])
        assert lat > 0
        name, plan = qs[i]
        got = cq.fetch_all(res)
        check(got, oracle_mod.query(tables[name][0], plan), f"query {i} ({name})")
        alone = cq.fetch_all(cq.cq_query_run(tables[name][1], plan))
        for a, b in zip(got, alone):
            assert np.array_equal(a, b)
    launches, completed = cq.cq_server_stats(srv)
    assert completed == len(qs) and 1 <= launches <= len(qs)
    srv.close()


def test_admission_and_errors(cq, ctx, tables):
    srv = cq.cq_server_create(ctx, cq.server_options(memory_budget_bytes=4096))
    with pytest.raises(cq.CQError) as e:                    # footprint above the whole budget
        cq.cq_server_submit(srv, tables["het"][1], tables["het_plan"])
    assert e.value.status == cq.CQ_ERR_BUSY
    with pytest.raises(cq.CQError) as e:                    # planning errors come back at submission
        cq.cq_server_submit(srv, tables["tiny"][1], dg.Plan([dg.Pred(7, "lt", 1)], [], [dg.Agg("count")]))
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
    with pytest.raises(cq.CQError) as e:
        cq.cq_server_wait(srv, 12345)
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
    srv.close()


def test_uncollected_results_and_released_handles(cq, ctx, oracle_mod):
    """The server holds what a queued query needs: the caller may drop its
    table and plan right after submitting, and may leave results uncollected."""
    srv = cq.cq_server_create(ctx)
    t, plan = dg.tiny_two_rle(50_000, seed=5)
    h, cols = cq.table_from(ctx, t)
    tickets = [cq.cq_server_submit(srv, h, dg.tiny_plan(k)) for k in (10, 50, 90)]
    h.close()
    for c in cols:
        c.close()
    res, _ = cq.cq_server_wait(srv, tickets[1])
    check(cq.fetch_all(res), oracle_mod.query(t, dg.tiny_plan(50)), "after release")
    srv.close()                                             # tickets 0 and 2 never collected
