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


def test_static_alignment_rejects_malformed_inputs():
    """Unsorted run ends, a last end other than n_rows, a capacity below the
    segment count and a row count near 2^64 (a negative size through the
    binding) are refused with their status; a good call still works after."""
    import torch

    from paper_2506_10092_gb300 import cq

    cq.cq_ctx_create(0)
    seg = torch.empty(64, dtype=torch.int64, device="cuda")
    ridx = torch.empty(128, dtype=torch.int64, device="cuda")

    def call(ends, n_rows, capacity=64):
        return cq.cq_align_segments_static(ends, n_rows, seg, ridx, capacity)

    good = [torch.tensor([3, 7, 10], dtype=torch.int64, device="cuda"),
            torch.tensor([5, 10], dtype=torch.int32, device="cuda")]
    with pytest.raises(cq.CQError) as e:
        call([torch.tensor([3, 2, 10], dtype=torch.int64, device="cuda")], 10)
    assert e.value.status == cq.CQ_ERR_UNSORTED
    with pytest.raises(cq.CQError) as e:
        call([torch.tensor([3, 7, 9], dtype=torch.int64, device="cuda")], 10)
    assert e.value.status == cq.CQ_ERR_SIZE_MISMATCH and "n_rows" in str(e.value)
    with pytest.raises(cq.CQError) as e:
        call(good, 10, capacity=3)          # segments end at 3, 5, 7, 10
    assert e.value.status == cq.CQ_ERR_SIZE_MISMATCH
    with pytest.raises(cq.CQError) as e:
        call(good, -1)
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
    assert call(good, 10) == 4
    torch.cuda.synchronize()
    assert seg[:4].tolist() == [3, 5, 7, 10]
    assert ridx[:4].tolist() == [0, 1, 1, 2]          # ridx[j * capacity + s]
    assert ridx[64:68].tolist() == [0, 0, 1, 1]
