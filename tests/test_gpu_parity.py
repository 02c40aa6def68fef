"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.  Every result of this method is
an exact integer (plus one correctly rounded division for AVG), so the bar is
bit-exact equality for keys, SUM, COUNT, MIN, MAX and AVG alike."""
import numpy as np
import pytest

from paper_2506_10092_gb300 import datagen as dg
from tests.helpers import random_column, random_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    from paper_2506_10092_gb300 import cq as _cq
    return _cq


@pytest.fixture(scope="module")
def ctx(cq):
    return cq.cq_ctx_create(0)


def run(cq, ctx, table, plan, device=False, opts=None):
    t, cols = cq.table_from(ctx, table, device=device)
    res = cq.cq_query_run(t, plan, opts=opts)
    return cq.fetch_all(res)


def check(got, ref, msg=""):
    want = ref.keys + ref.aggs
    assert len(got) == len(want), msg
    for i, (g, w) in enumerate(zip(got, want)):
        assert g.dtype == w.dtype, (msg, i, g.dtype, w.dtype)
        np.testing.assert_array_equal(g, w, err_msg=f"{msg} output column {i}")


# ------------------------------------------------------------------ the two workloads at test sizes
def test_tiny_two_rle_1m_rows(cq, ctx, oracle_mod):
    table, plan = dg.tiny_two_rle(1_000_000)
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), "tiny")


@pytest.mark.parametrize("device", [False, True])
def test_heterogeneous_2m_rows(cq, ctx, oracle_mod, device):
    table, plan = dg.heterogeneous(2_000_000 + 777, seed=3)     # ragged last tile
    check(run(cq, ctx, table, plan, device=device), oracle_mod.query(table, plan, n_threads=4), "hetero")


def test_heterogeneous_with_index_default_and_string_keys(cq, ctx, oracle_mod):
    table, plan = dg.heterogeneous(1_000_000, seed=5, index_default=-7)
    plan = dg.Plan(plan.preds, plan.group_by,
                   plan.aggs + [dg.Agg("avg", 2), dg.Agg("min", 2), dg.Agg("max", 2), dg.Agg("avg", 4),
                                dg.Agg("min", 1), dg.Agg("max", 0)])
    t, cols = cq.table_from(ctx, table)
    res = cq.cq_query_run(t, plan)
    got = cq.fetch_all(res)
    ref = oracle_mod.query(table, plan, n_threads=4)
    check(got, ref, "hetero+")
    strings = table.columns[1].strings
    for row in [0, len(got[0]) // 2, len(got[0]) - 1]:
        assert cq.cq_result_key_string(res, 1, row) == strings[int(got[1][row])]


# ------------------------------------------------------------------ random tables, every encoding
ENCS = ["rle", "plain", "packed", "index", "dict"]


@pytest.mark.parametrize("seed", range(60))
def test_random_tables(cq, ctx, oracle_mod, seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.choice([1, 31, 1000, 4095, 4096, 4097, 20000, 70001]))
    ncol = int(rng.integers(1, 5))
    cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(ncol)]
    table = dg.Table(cols, n)
    plan = random_plan(rng, table)
    ref = oracle_mod.query(table, plan)
    tile = int(rng.choice([1024, 2048, 4096, 8192]))
    opts = cq.exec_options(tile_rows=tile, stages=int(rng.choice([1, 2, 3, 4])),
                           table_slots=int(rng.choice([128, 1024])))
    check(run(cq, ctx, table, plan, device=bool(seed % 2), opts=opts), ref, f"seed {seed} tile {tile}")


@pytest.mark.parametrize("seed", range(12))
def test_decompress_then_scan_matches(cq, ctx, oracle_mod, seed):
    rng = np.random.default_rng(9000 + seed)
    n = int(rng.choice([100, 5000, 50001]))
    cols = [random_column(rng, n, str(rng.choice(ENCS))) for _ in range(3)]
    table = dg.Table(cols, n)
    plan = random_plan(rng, table)
    ref = oracle_mod.query(table, plan)
    check(run(cq, ctx, table, plan, opts=cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN)), ref, "dts")


# ------------------------------------------------------------------ segment-mode edge cases
def _rle(vals, ends, n, vt=np.int64, et=np.int64):
    return dg.RLE(np.asarray(vals, dtype=vt), np.asarray(ends, dtype=et), n)


@pytest.mark.parametrize("case", ["one_run", "unit_runs", "same_bounds", "tile_edges", "int32", "long_table"])
def test_rle_shapes(cq, ctx, oracle_mod, case):
    rng = np.random.default_rng(hash(case) % 1000)
    n = 50_000
    if case == "one_run":
        a = _rle([7], [n], n)
        b = dg.make_rle(rng, n, 3.0, 0, 9, np.int64, np.int64)
    elif case == "unit_runs":
        a = _rle(rng.integers(0, 5, n), np.arange(1, n + 1), n)
        b = _rle(rng.integers(0, 3, n), np.arange(1, n + 1), n)
    elif case == "same_bounds":
        ends = dg.geometric_ends(rng, n, 7.0, np.int64)
        a = _rle(rng.integers(0, 50, ends.shape[0]), ends, n)
        b = _rle(rng.integers(0, 4, ends.shape[0]), ends, n)
    elif case == "tile_edges":
        ends = np.arange(1024, n, 1024).tolist() + [n]
        a = _rle(rng.integers(0, 50, len(ends)), ends, n)
        b = _rle(rng.integers(0, 4, len(ends) + 1), sorted(set(ends + [4096 * 3 + 1])), n)
    elif case == "int32":
        a = dg.make_rle(rng, n, 4.0, -100, 100, np.int32, np.int32)
        b = dg.make_rle(rng, n, 2.0, 0, 20, np.int32, np.int32)
    else:
        n = 3_000_001
        a = dg.make_rle(rng, n, 30.0, 0, 99, np.int64, np.int64)
        b = dg.make_rle(rng, n, 300.0, 0, 9, np.int64, np.int64)
    table = dg.Table([a, b], n)
    plan = dg.Plan([dg.Pred(0, "lt", 25)], [1], [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 0),
                                                 dg.Agg("max", 0), dg.Agg("avg", 0)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), case)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_materialised_alignment(cq, ctx, oracle_mod, k):
    import torch
    rng = np.random.default_rng(k)
    n = 100_003
    cols = [dg.make_rle(rng, n, float(rng.choice([1.5, 6.0, 400.0])), 0, 9, np.int64,
                        np.int64 if j % 2 else np.int32) for j in range(k)]
    seg, ridx = oracle_mod.align([c.run_ends for c in cols], n)
    handles = [cq.column_from(ctx, c) for c in cols]
    S = cq.cq_align_segments(ctx, handles)
    assert S == seg.shape[0]
    d_seg = torch.empty(S, dtype=torch.int64, device="cuda")
    d_ridx = torch.empty(k * S, dtype=torch.int64, device="cuda")
    assert cq.cq_align_segments(ctx, handles, d_seg, d_ridx, S) == S
    np.testing.assert_array_equal(d_seg.cpu().numpy(), seg)
    np.testing.assert_array_equal(d_ridx.cpu().numpy().reshape(k, S), ridx)


# ------------------------------------------------------------------ packed widths and index density
@pytest.mark.parametrize("w", [1, 3, 7, 13, 20, 31, 32, 33, 47, 63, 64])
def test_bit_widths(cq, ctx, oracle_mod, w):
    rng = np.random.default_rng(w)
    n = 9000 + w
    off = rng.integers(0, 2**63, size=n, dtype=np.uint64) & np.uint64((1 << w) - 1 if w < 64 else 2**64 - 1)
    base = -(1 << 40) if w < 40 else 0
    p = dg.make_packed(off, w, base)
    key = dg.Plain(rng.integers(0, 3, n).astype(np.int64))
    table = dg.Table([p, key], n)
    plan = dg.Plan([dg.Pred(0, "ge", base + 1)], [1], [dg.Agg("min", 0), dg.Agg("max", 0), dg.Agg("count"),
                                                      dg.Agg("avg", 0)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), f"w={w}")


@pytest.mark.parametrize("nnz", ["zero", "all", "one"])
def test_index_density(cq, ctx, oracle_mod, nnz):
    rng = np.random.default_rng(11)
    n = 20_000
    k = {"zero": 0, "all": n, "one": 1}[nnz]
    x = dg.make_index(rng, n, k, -1000, 1000, default=5)
    key = dg.make_rle(rng, n, 100.0, 0, 4, np.int64, np.int64)
    table = dg.Table([x, key], n)
    plan = dg.Plan([], [1], [dg.Agg("sum", 0), dg.Agg("min", 0), dg.Agg("max", 0), dg.Agg("count")])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), nnz)
    plan = dg.Plan([dg.Pred(0, "ne", 5)], [0], [dg.Agg("count")])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan), nnz + " key")


# ------------------------------------------------------------------ degenerate plans and errors
def test_no_group_by_nothing_passes(cq, ctx, oracle_mod):
    table, plan = dg.tiny_two_rle(10_000)
    plan = dg.Plan([dg.Pred(0, "lt", -1)], [], [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 0),
                                                dg.Agg("avg", 0)])
    got = run(cq, ctx, table, plan)
    check(got, oracle_mod.query(table, plan), "empty")
    assert got[1][0] == 0


def test_in_list_with_unknown_strings(cq, ctx, oracle_mod):
    table, plan = dg.heterogeneous(300_000, seed=9)
    plan = dg.Plan([dg.Pred(1, "in", strs=[b"not-a-word", b"zzzz"])], [0], [dg.Agg("count")])
    got = run(cq, ctx, table, plan)
    check(got, oracle_mod.query(table, plan), "unknown")
    assert len(got[0]) == 0


def test_sum_overflow_is_an_error(cq, ctx):
    big = 2**62 + 1
    table = dg.Table([_rle([big, big], [3, 5], 5)], 5)
    t, cols = cq.table_from(ctx, table)
    res = cq.cq_query_run(t, dg.Plan([], [], [dg.Agg("sum", 0)]))
    with pytest.raises(cq.CQError) as e:
        cq.cq_result_wait(res)
    assert e.value.status == cq.CQ_ERR_OVERFLOW
    # AVG of the same values is still exact
    res = cq.cq_query_run(t, dg.Plan([], [], [dg.Agg("avg", 0)]))
    assert cq.fetch_all(res)[0][0] == float(5 * big) / 5.0


@pytest.mark.parametrize("bad", ["unsorted", "short", "pos_range", "code_range", "few_words"])
def test_malformed_columns_rejected(cq, ctx, bad):
    n = 10
    with pytest.raises(cq.CQError) as e:
        if bad == "unsorted":
            cq.cq_column_create_rle(ctx, np.array([1, 2]), np.array([6, 4]), n)
        elif bad == "short":
            cq.cq_column_create_rle(ctx, np.array([1, 2]), np.array([4, 9]), n)
        elif bad == "pos_range":
            cq.cq_column_create_index(ctx, np.array([1]), np.array([10]), 0, n)
        elif bad == "code_range":
            cq.column_from(ctx, dg.make_dict([b"x", b"y", b"z"], np.full(n, 3, dtype=np.uint64), 2))
        else:
            cq.cq_column_create_bitpacked(ctx, np.zeros(2, dtype=np.uint32), 7, 0, n)
    assert e.value.status in (cq.CQ_ERR_UNSORTED, cq.CQ_ERR_SIZE_MISMATCH, cq.CQ_ERR_INVALID_ARG)


def test_repeat_runs_are_deterministic(cq, ctx):
    table, plan = dg.heterogeneous(500_000, seed=1)
    t, cols = cq.table_from(ctx, table)
    a = cq.fetch_all(cq.cq_query_run(t, plan))
    b = cq.fetch_all(cq.cq_query_run(t, plan))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


# ------------------------------------------------------------------ many tiles per CTA
@pytest.mark.parametrize("ctas", [1, 2])
@pytest.mark.parametrize("grid,tile,slots", [(1, 1024, 128), (3, 4096, 1024), (7, 2048, 256), (16, 8192, 0)])
def test_many_tiles_per_cta_heterogeneous(cq, ctx, oracle_mod, grid, tile, slots, ctas):
    """Few CTAs walk many tiles each: bulk-copy stages are reused, run and
    position cursors carry across tiles and the group table flushes often."""
    table, plan = dg.heterogeneous(3_000_000 + 123, seed=21, index_default=3)
    ref = oracle_mod.query(table, plan, n_threads=4)
    opts = cq.exec_options(tile_rows=tile, grid_ctas=grid, table_slots=slots, ctas_per_sm=ctas)
    check(run(cq, ctx, table, plan, opts=opts), ref, f"grid {grid} ctas/SM {ctas}")


@pytest.mark.parametrize("grid", [1, 5])
def test_many_tiles_per_cta_segments(cq, ctx, oracle_mod, grid):
    table, plan = dg.tiny_two_rle(1_000_000, seed=3)
    plan = dg.Plan(plan.preds, [1, 0], plan.aggs + [dg.Agg("max", 0)])
    ref = oracle_mod.query(table, plan)
    check(run(cq, ctx, table, plan, opts=cq.exec_options(grid_ctas=grid, tile_rows=1024)), ref, f"seg grid {grid}")


@pytest.mark.parametrize("tile,ctas", [(2048, 2), (4096, 2), (4096, 1), (8192, 1)])
def test_heterogeneous_20m_rows_all_tiles(cq, ctx, oracle_mod, tile, ctas):
    """20M rows: every CTA walks many tiles at every tile size (this shape
    once exposed a device-side key error at 8192-row tiles)."""
    table, plan = dg.heterogeneous(20_000_000, seed=20250611)
    ref = oracle_mod.query(table, plan, n_threads=oracle_mod.cores())
    check(run(cq, ctx, table, plan, opts=cq.exec_options(tile_rows=tile, ctas_per_sm=ctas)), ref, f"20M tile {tile}")


@pytest.mark.parametrize("seg", [False, True])
def test_single_group_queries(cq, ctx, oracle_mod, seg):
    """No GROUP BY: every passing item lands in one group (warp-reduced path)."""
    table, plan = dg.heterogeneous(1_000_000, seed=12) if not seg else dg.tiny_two_rle(1_000_000, seed=12)
    if not seg:
        plan = dg.Plan(plan.preds, [], [dg.Agg("sum", 4), dg.Agg("min", 4), dg.Agg("max", 4), dg.Agg("count"),
                                         dg.Agg("sum", 3), dg.Agg("avg", 2), dg.Agg("max", 0)])
    else:
        plan = dg.Plan(plan.preds, [], [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 1), dg.Agg("avg", 0)])
    check(run(cq, ctx, table, plan), oracle_mod.query(table, plan, n_threads=4), f"one group seg={seg}")


# ------------------------------------------------------------------ long aligned segments (segment mode)
@pytest.mark.parametrize("case", ["long_runs", "one_run_each", "ends_on_tile_edges", "sparse_index", "no_keys",
                                  "mixed_lengths"])
@pytest.mark.parametrize("tile,kernel", [(4096, 2), (8192, 2), (8192, 3)])
def test_long_segments(cq, ctx, oracle_mod, case, tile, kernel):
    """Segment mode aggregates a stretch without boundaries in any column once
    (value x length) and skips its tiles.  Runs far longer than a tile, runs
    ending exactly on tile edges, a sparse index column cutting the stretches,
    a plan without GROUP BY, and long runs mixed with short ones: every result
    equals the oracle's."""
    rng = np.random.default_rng(abs(hash(case)) % 10_000 + tile)
    n = 3_000_017
    if case == "long_runs":
        cols = [dg.make_rle(rng, n, 40_000.0, 0, 99, np.int64, np.int64),
                dg.make_rle(rng, n, 90_000.0, 0, 9, np.int32, np.int32)]
    elif case == "one_run_each":
        cols = [_rle([42], [n], n), _rle([3], [n], n)]
    elif case == "ends_on_tile_edges":
        e1 = sorted(set(list(range(8192 * 3, n, 8192 * 7)) + [n]))
        e2 = sorted(set(list(range(4096 * 5, n, 4096 * 11)) + [n]))
        cols = [_rle(rng.integers(0, 99, len(e1)), e1, n), _rle(rng.integers(0, 9, len(e2)), e2, n)]
    elif case == "sparse_index":
        pos = np.sort(rng.choice(n, size=40, replace=False)).astype(np.int64)
        cols = [dg.make_rle(rng, n, 100_000.0, 0, 99, np.int64, np.int64),
                dg.Index(rng.integers(-5, 5, size=40).astype(np.int64), pos, 7, n)]
    elif case == "no_keys":
        cols = [dg.make_rle(rng, n, 60_000.0, 0, 99, np.int64, np.int64),
                dg.make_rle(rng, n, 25_000.0, 0, 9, np.int64, np.int64)]
    else:
        cols = [dg.make_rle(rng, n, 50_000.0, 0, 99, np.int64, np.int64),
                dg.make_rle(rng, n, 2.0, 0, 9, np.int64, np.int64)]
    table = dg.Table(cols, n)
    gb = [] if case == "no_keys" else [1]
    plan = dg.Plan([dg.Pred(0, "lt", 60)], gb, [dg.Agg("sum", 0), dg.Agg("count"), dg.Agg("min", 1), dg.Agg("max", 0),
                                               dg.Agg("avg", 1)])
    ref = oracle_mod.query(table, plan)
    check(run(cq, ctx, table, plan, opts=cq.exec_options(tile_rows=tile, kernel=kernel)), ref,
          f"{case} tile {tile} kernel {kernel}")
    # and as one query of a batch (the persistent kernel's tile walk)
    t, _cols = cq.table_from(ctx, table)
    res = cq.cq_batch_run([t, t], [plan, plan])
    for r in res:
        check(cq.fetch_all(r), ref, f"{case} batched")


@pytest.mark.parametrize("seed", range(24))
def test_segment_mode_walks_agree(cq, ctx, oracle_mod, seed):
    """Random all-RLE / index tables (run lengths from 1.5 to 5e4 rows, index
    columns from empty to dense, int32 and int64) walked tile by tile and run
    by run: both equal the oracle."""
    rng = np.random.default_rng(11_000 + seed)
    n = int(rng.choice([1, 777, 8192, 100_001, 1_000_003]))
    cols = []
    for _ in range(int(rng.integers(1, 4))):
        if rng.random() < 0.7:
            dt = np.int64 if rng.random() < 0.5 else np.int32
            cols.append(dg.make_rle(rng, n, float(rng.choice([1.5, 7.0, 300.0, 5e4])), -20, 20, dt, dt))
        else:
            nnz = int(rng.choice([0, 1, max(1, n // 1000), n // 3, n]))
            pos = np.sort(rng.choice(n, size=nnz, replace=False)).astype(np.int64)
            cols.append(dg.Index(rng.integers(-20, 20, size=nnz).astype(np.int64), pos, int(rng.integers(-3, 3)), n))
    table = dg.Table(cols, n)
    plan = random_plan(rng, table)
    ref = oracle_mod.query(table, plan)
    for kernel in (2, 3):
        check(run(cq, ctx, table, plan, opts=cq.exec_options(kernel=kernel)), ref, f"seed {seed} kernel {kernel}")
