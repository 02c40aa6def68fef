"""The allocation-free alignment entry point against the allocating one.

cq_align_segments_static serves callers that cannot allocate device memory
while they run (a memory budget owned by someone else, a pre-sized arena):
it keeps its scratch in a fixed array inside the library.  Its segments and
run indices must equal those of cq_align_segments, call after call -- the
shared array keeps the previous call's contents, so two different inputs are
aligned back to back.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


def test_static_alignment_matches_the_allocating_entry_point():
    import torch

    from paper_2506_10092_gb300 import cq

    ctx = cq.cq_ctx_create(0)
    rng = np.random.default_rng(2026)
    shapes = [(300_007, [1.5, 40.0, 6.0], [np.int64, np.int32, np.int64]),
              (123_457, [3.0, 900.0], [np.int32, np.int32])]
    for n, means, dts in shapes:                   # two calls in a row, different inputs
        cols = [dg.make_rle(rng, n, m, 0, 9, np.int64, dt) for m, dt in zip(means, dts)]
        k = len(cols)
        handles = [cq.column_from(ctx, c) for c in cols]
        S = cq.cq_align_segments(ctx, handles)
        seg_a = torch.empty(S, dtype=torch.int64, device="cuda")
        ridx_a = torch.empty(k * S, dtype=torch.int64, device="cuda")
        assert cq.cq_align_segments(ctx, handles, seg_a, ridx_a, S) == S

        ends = [torch.from_numpy(np.ascontiguousarray(c.run_ends)).cuda() for c in cols]
        assert cq.cq_align_segments_static(ends, n) == S
        seg_b = torch.full((S,), -1, dtype=torch.int64, device="cuda")
        ridx_b = torch.full((k * S,), -1, dtype=torch.int64, device="cuda")
        assert cq.cq_align_segments_static(ends, n, seg_b, ridx_b, S) == S
        torch.cuda.synchronize()
        assert torch.equal(seg_a, seg_b)
        assert torch.equal(ridx_a, ridx_b)

    # sizes beyond the fixed scratch are refused before any device work
    with pytest.raises(cq.CQError) as e:
        cq.cq_align_segments_static(ends, 65536 * 4096 + 1)
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
