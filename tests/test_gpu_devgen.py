"""The device-side generator of the nested table against the host-side one:
the same packed words, bit for bit, so that the oracle (fed by the host
generator) and the CUDA path (fed by the device generator) see one table."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 8, 1000, 65_537, 1_000_003])
@pytest.mark.parametrize("w,col", [(8, 7), (12, 8), (16, 6), (8, 5), (1, 9), (32, 3)])
def test_hash_fields_match_host(n, w, col):
    from paper_2506_10092_gb300 import devgen
    dev = devgen.hash_fields(n, w, 12345, col).cpu().numpy().view(np.uint32)
    rows = np.arange(n, dtype=np.uint64)
    vals = (dg.splitmix64(12345, col, rows) & np.uint64((1 << w) - 1)).astype(np.uint64)
    assert np.array_equal(dev, dg.pack_bits(vals, w))


@pytest.mark.parametrize("n", [1, 9, 4096, 300_001])
def test_nested_codes_match_host(n):
    import torch
    from paper_2506_10092_gb300 import devgen
    _, _, c3 = dg.nested_runs(n, seed=8)
    ends = torch.from_numpy(c3.run_ends.astype(np.int64)).cuda()
    dev = devgen.nested_codes4(ends, n, 8).cpu().numpy().view(np.uint32)
    assert np.array_equal(dev, dg.pack_bits(dg.nested_codes4_all(8, c3.run_ends, n), 4))


def test_device_nested_table_matches_oracle(oracle_mod):
    from paper_2506_10092_gb300 import cq, devgen
    ctx = cq.cq_ctx_create(0)
    t = devgen.DeviceNested(cq, ctx, 2_000_003, seed=31)
    host = t.host_table()
    for lo, hi in [(200, 699), (0, 999), (500, 500)]:
        plan = dg.nested_plan(lo, hi, lean=True)
        got = cq.fetch_all(cq.cq_query_run(t.table, plan))
        ref = oracle_mod.query(host, plan, n_threads=4)
        for g, r in zip(got, ref.keys + ref.aggs):
            np.testing.assert_array_equal(g, r)
