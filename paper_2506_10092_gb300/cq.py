"""Thin Python binding of the cq C ABI (include/cq.h).

Argument marshalling only: every step of a query runs in the CUDA library
``libcq.so``.  Function names are the C names.  Buffers may be numpy arrays
(host memory, copied by the library) or CUDA torch tensors (device memory,
borrowed: the Python column object keeps them alive).

Importing this module loads the library and raises ``ImportError`` when it
is missing; there is no fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import datagen as dg

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcq.so")

CQ_OK = 0
CQ_ERR_INVALID_ARG, CQ_ERR_UNSORTED, CQ_ERR_SIZE_MISMATCH, CQ_ERR_OOM, CQ_ERR_CUDA = -1, -2, -3, -4, -5
CQ_ERR_OVERFLOW, CQ_ERR_UNSUPPORTED, CQ_ERR_TABLE_FULL, CQ_ERR_TIMEOUT, CQ_ERR_NOT_READY, CQ_ERR_BUSY = \
    -6, -7, -8, -9, -10, -11
CQ_I32, CQ_I64 = 1, 2
CQ_MEM_HOST_COPY, CQ_MEM_DEVICE_BORROW = 0, 1
CQ_EXEC_FUSED, CQ_EXEC_DECOMPRESS_THEN_SCAN = 0, 1
OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7}
AGGS = {"sum": 0, "count": 1, "min": 2, "max": 3, "avg": 4, "var_pop": 5, "var_samp": 6, "std_pop": 7,
        "std_samp": 8}


class CQError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"cq status {status}: {message}")
        self.status = status


class cq_predicate(C.Structure):
    _fields_ = [("col", C.c_uint32), ("op", C.c_int32), ("lo", C.c_int64), ("hi", C.c_int64),
                ("in_ints", C.c_void_p), ("n_in", C.c_uint32),
                ("strs", C.c_void_p), ("str_lens", C.c_void_p), ("n_strs", C.c_uint32),
                ("or_group", C.c_uint32), ("negate", C.c_uint32)]


class cq_filter_node(C.Structure):
    _fields_ = [("kind", C.c_int32), ("arg", C.c_uint32)]


CQ_NODE_PRED, CQ_NODE_AND, CQ_NODE_OR, CQ_NODE_NOT = 0, 1, 2, 3
NODES = {"pred": CQ_NODE_PRED, "and": CQ_NODE_AND, "or": CQ_NODE_OR, "not": CQ_NODE_NOT}


class cq_aggregate(C.Structure):
    _fields_ = [("op", C.c_int32), ("col", C.c_uint32), ("expr", C.c_int32), ("col2", C.c_uint32)]


EXPRS = {None: 0, "add": 1, "sub": 2, "mul": 3}   # cq_expr


class cq_plan(C.Structure):
    _fields_ = [("preds", C.c_void_p), ("n_preds", C.c_uint32),
                ("group_by", C.c_void_p), ("n_group_by", C.c_uint32),
                ("aggs", C.c_void_p), ("n_aggs", C.c_uint32),
                ("filter", C.c_void_p), ("n_filter", C.c_uint32)]


class cq_exec_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile_rows", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("stages", C.c_uint32), ("table_slots", C.c_uint32), ("grid_ctas", C.c_uint32),
                ("items_per_cta", C.c_uint32), ("kernel", C.c_uint32),
                ("hash_slots_log2", C.c_uint32)]


class cq_server_options(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_uint64), ("max_batch", C.c_uint32), ("n_streams", C.c_uint32),
                ("max_wait_us", C.c_uint32), ("large_rows_log2", C.c_uint32), ("reserved", C.c_uint32 * 2)]


_VP = C.c_void_p
_SIGS = {
    "cq_ctx_create": [C.c_int, _VP, C.POINTER(_VP)],
    "cq_ctx_destroy": [_VP],
    "cq_ctx_num_sms": [_VP, C.POINTER(C.c_uint32)],
    "cq_last_error": [],
    "cq_column_create_rle": [_VP, C.c_int, _VP, C.c_int, _VP, C.c_uint64, C.c_uint64, C.c_uint32, C.POINTER(_VP)],
    "cq_column_create_rle_index": [_VP, C.c_int, C.c_int, _VP, _VP, _VP, C.c_uint64, _VP, _VP, C.c_uint64,
                                   C.c_uint64, C.POINTER(_VP)],
    "cq_column_create_dict": [_VP, _VP, _VP, C.c_uint32, _VP, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32,
                              C.POINTER(_VP)],
    "cq_column_create_index": [_VP, C.c_int, _VP, C.c_int, _VP, C.c_uint64, C.c_int64, C.c_uint64, C.c_uint32,
                               C.POINTER(_VP)],
    "cq_column_create_bitpacked": [_VP, C.c_int, _VP, C.c_uint64, C.c_uint32, C.c_int64, C.c_uint64, C.c_uint32,
                                   C.POINTER(_VP)],
    "cq_column_create_plain": [_VP, C.c_int, _VP, C.c_uint64, C.c_uint32, C.POINTER(_VP)],
    "cq_column_destroy": [_VP],
    "cq_column_encoding": [_VP, C.POINTER(C.c_uint32)],
    "cq_column_device_bytes": [_VP, C.POINTER(C.c_uint64)],
    "cq_table_bind": [_VP, _VP, C.c_uint32, C.POINTER(_VP)],
    "cq_table_destroy": [_VP],
    "cq_table_num_rows": [_VP, C.POINTER(C.c_uint64)],
    "cq_filter_conjunctive": [C.POINTER(cq_plan), _VP, C.c_uint32, C.POINTER(C.c_uint32)],
    "cq_query_run": [_VP, C.POINTER(cq_plan), _VP, C.POINTER(_VP)],
    "cq_query_run_ex": [_VP, C.POINTER(cq_plan), C.POINTER(cq_exec_options), _VP, C.POINTER(_VP)],
    "cq_batch_run": [C.c_uint32, _VP, _VP, C.POINTER(cq_exec_options), _VP, _VP],
    "cq_batch_tune": [C.c_uint32, _VP, _VP, _VP, C.POINTER(cq_exec_options), C.POINTER(C.c_double)],
    "cq_result_wait": [_VP, C.c_uint64],
    "cq_result_num_groups": [_VP, C.POINTER(C.c_uint64)],
    "cq_result_num_columns": [_VP, C.POINTER(C.c_uint32)],
    "cq_result_column_kind": [_VP, C.c_uint32, C.POINTER(C.c_uint32)],
    "cq_result_fetch": [_VP, C.c_uint32, _VP, C.c_uint64],
    "cq_result_device_column": [_VP, C.c_uint32, C.POINTER(_VP)],
    "cq_result_key_string": [_VP, C.c_uint32, C.c_uint64, C.POINTER(C.c_char_p), C.POINTER(C.c_uint32)],
    "cq_result_device_time_us": [_VP, C.POINTER(C.c_double)],
    "cq_result_kernel_time_us": [_VP, C.POINTER(C.c_double)],
    "cq_result_destroy": [_VP],
    "cq_align_segments": [_VP, _VP, C.c_uint32, _VP, _VP, _VP, C.c_uint64, C.POINTER(C.c_uint64)],
    "cq_align_segments_static": [C.c_uint32, _VP, _VP, _VP, C.c_uint64, _VP, _VP, _VP, C.c_uint64,
                                 C.POINTER(C.c_uint64)],
    "cq_server_create": [_VP, C.POINTER(cq_server_options), C.POINTER(_VP)],
    "cq_server_submit": [_VP, _VP, C.POINTER(cq_plan), C.POINTER(C.c_uint64)],
    "cq_server_wait": [_VP, C.c_uint64, C.c_uint64, C.POINTER(_VP), C.POINTER(C.c_double)],
    "cq_server_stats": [_VP, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
    "cq_server_destroy": [_VP],
    "cq_selftest_bounded_wait": [_VP, C.c_uint32, C.POINTER(C.c_int32)],
    "cq_jit_stats": [C.POINTER(C.c_uint64), C.POINTER(C.c_double)],
    "cq_jit_check": [C.c_uint32, C.POINTER(C.c_double)],
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcq.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_char_p if name == "cq_last_error" else C.c_int
    return lib


lib = _load()


def _check(rc: int):
    if rc != CQ_OK:
        raise CQError(rc, lib.cq_last_error().decode(errors="replace"))
    return rc


def _dt(a) -> int:
    s = str(a.dtype)
    if s.endswith("int64"):
        return CQ_I64
    if s.endswith("int32"):
        return CQ_I32
    raise TypeError(f"unsupported dtype {a.dtype}")


def _is_dev(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a):
    if a is None:
        return None
    if _is_dev(a) or hasattr(a, "data_ptr"):     # CUDA tensor, or a (pinned) host tensor
        return a.data_ptr() if a.numel() else None
    return a.ctypes.data if a.size else None


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- handles
_EXITING = False


def _at_exit():
    # the process is ending: leave handles to the driver instead of calling
    # into CUDA while the interpreter (and torch) tear down in any order
    global _EXITING
    _EXITING = True


atexit.register(_at_exit)


class Handle:
    def __init__(self, ptr, destroy, keep=()):
        self.ptr = ptr
        self._destroy = destroy
        self.keep = list(keep)

    def close(self):
        if self.ptr and not _EXITING:
            self._destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cq_ctx_create(device: int = 0, stream=None) -> Handle:
    out = C.c_void_p()
    _check(lib.cq_ctx_create(device, _stream_ptr(stream), C.byref(out)))
    return Handle(out.value, lib.cq_ctx_destroy)


def cq_ctx_num_sms(ctx) -> int:
    n = C.c_uint32()
    _check(lib.cq_ctx_num_sms(ctx.ptr, C.byref(n)))
    return n.value


def _mem(*arrays) -> int:
    dev = [_is_dev(a) for a in arrays if a is not None]
    if any(dev) and not all(dev):
        raise ValueError("mix of host and device buffers")
    return CQ_MEM_DEVICE_BORROW if dev and dev[0] else CQ_MEM_HOST_COPY


def _contig(a):
    if a is None:
        return None
    if _is_dev(a):
        return a.contiguous()
    return np.ascontiguousarray(a)


def cq_column_create_rle(ctx, run_values, run_ends, n_rows: int) -> Handle:
    v, e = _contig(run_values), _contig(run_ends)
    out = C.c_void_p()
    _check(lib.cq_column_create_rle(ctx.ptr, _dt(v), _ptr(v), _dt(e), _ptr(e), int(e.shape[0]), int(n_rows),
                                    _mem(v, e), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx] + ([v, e] if _is_dev(v) else []))


def cq_column_create_rle_index(ctx, run_values, run_starts, run_ends, values, positions, n_rows: int) -> Handle:
    """Host arrays; values share one dtype, starts / ends / positions another."""
    rv = np.ascontiguousarray(run_values)
    vv = np.ascontiguousarray(values, dtype=rv.dtype)
    rs = np.ascontiguousarray(run_starts)
    re_ = np.ascontiguousarray(run_ends, dtype=rs.dtype)
    ps = np.ascontiguousarray(positions, dtype=rs.dtype)
    out = C.c_void_p()
    _check(lib.cq_column_create_rle_index(ctx.ptr, _dt(rv), _dt(rs), _ptr(rv), _ptr(rs), _ptr(re_), int(rs.shape[0]),
                                          _ptr(vv), _ptr(ps), int(ps.shape[0]), int(n_rows), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx])


def cq_column_create_dict(ctx, strings: Sequence[bytes], packed_codes, bit_width: int, n_rows: int) -> Handle:
    w = _contig(packed_codes)
    blob = b"".join(strings)
    offs = np.zeros(len(strings) + 1, dtype=np.uint64)
    np.cumsum([len(s) for s in strings], out=offs[1:]) if strings else None
    bb = C.create_string_buffer(blob, max(1, len(blob)))
    out = C.c_void_p()
    n_words = int(w.shape[0]) if not _is_dev(w) else int(w.numel())
    _check(lib.cq_column_create_dict(ctx.ptr, C.addressof(bb), offs.ctypes.data, len(strings), _ptr(w), n_words,
                                     int(bit_width), int(n_rows), _mem(w), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx] + ([w] if _is_dev(w) else []))


def cq_column_create_index(ctx, values, positions, default_value: int, n_rows: int) -> Handle:
    v, p = _contig(values), _contig(positions)
    out = C.c_void_p()
    _check(lib.cq_column_create_index(ctx.ptr, _dt(v), _ptr(v), _dt(p), _ptr(p), int(p.shape[0]),
                                      int(default_value), int(n_rows), _mem(v, p), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx] + ([v, p] if _is_dev(v) else []))


def cq_column_create_bitpacked(ctx, words, bit_width: int, base: int, n_rows: int, logical=CQ_I64) -> Handle:
    w = _contig(words)
    out = C.c_void_p()
    n_words = int(w.shape[0]) if not _is_dev(w) else int(w.numel())
    _check(lib.cq_column_create_bitpacked(ctx.ptr, logical, _ptr(w), n_words, int(bit_width), int(base),
                                          int(n_rows), _mem(w), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx] + ([w] if _is_dev(w) else []))


def cq_column_create_plain(ctx, values) -> Handle:
    v = _contig(values)
    out = C.c_void_p()
    _check(lib.cq_column_create_plain(ctx.ptr, _dt(v), _ptr(v), int(v.shape[0]), _mem(v), C.byref(out)))
    return Handle(out.value, lib.cq_column_destroy, [ctx] + ([v] if _is_dev(v) else []))


def cq_column_encoding(col) -> int:
    e = C.c_uint32()
    _check(lib.cq_column_encoding(col.ptr, C.byref(e)))
    return e.value


def cq_column_device_bytes(col) -> int:
    n = C.c_uint64()
    _check(lib.cq_column_device_bytes(col.ptr, C.byref(n)))
    return n.value


def cq_table_bind(ctx, cols: Sequence[Handle]) -> Handle:
    arr = (C.c_void_p * len(cols))(*[c.ptr for c in cols])
    out = C.c_void_p()
    _check(lib.cq_table_bind(ctx.ptr, C.addressof(arr), len(cols), C.byref(out)))
    return Handle(out.value, lib.cq_table_destroy, [ctx] + list(cols))


# ---------------------------------------------------------------- plans
class PlanStruct:
    """A cq_plan plus every buffer it points to."""

    def __init__(self, plan: dg.Plan):
        self.keep = []
        preds = (cq_predicate * max(1, len(plan.preds)))()
        for i, p in enumerate(plan.preds):
            s = preds[i]
            s.col, s.op, s.lo, s.hi = int(p.col), OPS[p.op], int(p.lo), int(p.hi)
            s.or_group, s.negate = int(getattr(p, "group", 0)), 1 if getattr(p, "neg", False) else 0
            if p.ints is not None:
                a = np.ascontiguousarray(np.asarray(list(p.ints), dtype=np.int64))
                self.keep.append(a)
                s.in_ints, s.n_in = (a.ctypes.data if a.size else None), int(a.shape[0])
            if p.strs is not None:
                bufs = [C.create_string_buffer(bytes(x), len(x) + 1) for x in p.strs]
                ptrs = (C.c_void_p * max(1, len(bufs)))(*[C.addressof(b) for b in bufs])
                lens = np.array([len(x) for x in p.strs] or [0], dtype=np.uint32)
                self.keep += [bufs, ptrs, lens]
                s.strs, s.str_lens, s.n_strs = C.addressof(ptrs), lens.ctypes.data, len(bufs)
        gb = np.array(list(plan.group_by) or [0], dtype=np.uint32)
        aggs = (cq_aggregate * max(1, len(plan.aggs)))(*[cq_aggregate(AGGS[a.op], int(a.col),
                                                                      EXPRS[getattr(a, "expr", None)],
                                                                      int(getattr(a, "col2", 0)))
                                                         for a in plan.aggs])
        prog = list(getattr(plan, "filter", None) or [])
        nodes = (cq_filter_node * max(1, len(prog)))(*[cq_filter_node(NODES[k], int(a)) for k, a in prog])
        self.keep += [preds, gb, aggs, nodes]
        self.s = cq_plan(C.addressof(preds), len(plan.preds), gb.ctypes.data, len(plan.group_by),
                         C.addressof(aggs), len(plan.aggs), C.addressof(nodes) if prog else None, len(prog))
        self.plan = plan


KERNEL_SPECIALISED, KERNEL_GENERIC = 0, 1


def exec_options(mode=CQ_EXEC_FUSED, tile_rows=0, ctas_per_sm=0, stages=0, table_slots=0,
                 grid_ctas=0, items_per_cta=0, kernel=KERNEL_SPECIALISED, hash_slots_log2=0) -> cq_exec_options:
    o = cq_exec_options()
    o.mode, o.tile_rows, o.ctas_per_sm, o.stages, o.table_slots = mode, tile_rows, ctas_per_sm, stages, table_slots
    o.grid_ctas, o.items_per_cta, o.kernel, o.hash_slots_log2 = grid_ctas, items_per_cta, kernel, hash_slots_log2
    return o


def cq_filter_conjunctive(plan: dg.Plan):
    """The conjunctive form of a plan's filter (host only): a list of
    (index of the plan predicate it copies, or_group, negate); the copies
    are matched to the plan's predicates by identity of their fields."""
    ps = PlanStruct(plan)
    cap = 16
    out = (cq_predicate * cap)()
    n = C.c_uint32()
    _check(lib.cq_filter_conjunctive(C.byref(ps.s), C.addressof(out), cap, C.byref(n)))
    src = (cq_predicate * max(1, len(plan.preds))).from_address(ps.s.preds)
    res = []
    for i in range(n.value):
        o = out[i]
        idx = next(j for j in range(len(plan.preds))
                   if (src[j].col, src[j].op, src[j].lo, src[j].hi, src[j].in_ints, src[j].strs)
                   == (o.col, o.op, o.lo, o.hi, o.in_ints, o.strs))
        res.append((idx, int(o.or_group), int(o.negate)))
    return res


def cq_jit_check(variant: int) -> float:
    """Compile (no GPU needed) one of the built-in check shapes; returns seconds."""
    sec = C.c_double()
    _check(lib.cq_jit_check(variant, C.byref(sec)))
    return sec.value


def cq_jit_stats():
    """(kernels compiled at run time by this process, seconds spent compiling)."""
    n, sec = C.c_uint64(), C.c_double()
    _check(lib.cq_jit_stats(C.byref(n), C.byref(sec)))
    return n.value, sec.value


class _Batch:
    """The cq_table* / cq_plan arrays of one batch call."""

    def __init__(self, tables, plans):
        if len(tables) != len(plans):
            raise ValueError("one plan per table")
        self.plans = [p if isinstance(p, PlanStruct) else PlanStruct(p) for p in plans]
        self.tables = list(tables)
        self.n = len(self.tables)
        self.tarr = (C.c_void_p * max(1, self.n))(*[t.ptr for t in self.tables])
        self.parr = (cq_plan * max(1, self.n))(*[ps.s for ps in self.plans])


def cq_batch_run(tables, plans, stream=None, opts: Optional[cq_exec_options] = None) -> list:
    """Run query i = (tables[i], plans[i]) for every i as one persistent launch;
    returns one result handle per query."""
    b = _Batch(tables, plans)
    out = (C.c_void_p * max(1, b.n))()
    _check(lib.cq_batch_run(b.n, C.addressof(b.tarr), C.addressof(b.parr),
                            C.byref(opts) if opts is not None else None, _stream_ptr(stream), C.addressof(out)))
    return [Handle(out[i], lib.cq_result_destroy, [b.tables[i], b.plans[i]]) for i in range(b.n)]


def cq_batch_tune(tables, plans, stream=None):
    """Autotune the batch shape; returns (cq_exec_options, launch microseconds)."""
    b = _Batch(tables, plans)
    best = cq_exec_options()
    us = C.c_double()
    _check(lib.cq_batch_tune(b.n, C.addressof(b.tarr), C.addressof(b.parr), _stream_ptr(stream),
                             C.byref(best), C.byref(us)))
    return best, us.value


def cq_query_run(table, plan, stream=None, opts: Optional[cq_exec_options] = None) -> Handle:
    ps = plan if isinstance(plan, PlanStruct) else PlanStruct(plan)
    out = C.c_void_p()
    if opts is None:
        _check(lib.cq_query_run(table.ptr, C.byref(ps.s), _stream_ptr(stream), C.byref(out)))
    else:
        _check(lib.cq_query_run_ex(table.ptr, C.byref(ps.s), C.byref(opts), _stream_ptr(stream), C.byref(out)))
    return Handle(out.value, lib.cq_result_destroy, [table, ps])


cq_query_run_ex = cq_query_run


def cq_selftest_bounded_wait(ctx, limit_us: int) -> int:
    """Device status left by a bounded wait on a barrier nothing completes."""
    st = C.c_int32()
    _check(lib.cq_selftest_bounded_wait(ctx.ptr, limit_us, C.byref(st)))
    return st.value


# ---------------------------------------------------------------- serving loop
def server_options(memory_budget_bytes=0, max_batch=0, n_streams=0, max_wait_us=0,
                   large_rows_log2=0) -> cq_server_options:
    o = cq_server_options()
    o.memory_budget_bytes, o.max_batch, o.n_streams, o.max_wait_us = memory_budget_bytes, max_batch, n_streams, \
        max_wait_us
    o.large_rows_log2 = large_rows_log2
    return o


def cq_server_create(ctx, opts: Optional[cq_server_options] = None) -> Handle:
    out = C.c_void_p()
    _check(lib.cq_server_create(ctx.ptr, C.byref(opts) if opts is not None else None, C.byref(out)))
    return Handle(out.value, lib.cq_server_destroy, [ctx])


def cq_server_submit(srv, table, plan) -> int:
    ps = plan if isinstance(plan, PlanStruct) else PlanStruct(plan)
    t = C.c_uint64()
    _check(lib.cq_server_submit(srv.ptr, table.ptr, C.byref(ps.s), C.byref(t)))
    return t.value


def cq_server_wait(srv, ticket: int, timeout_us: int = 2**64 - 1):
    """Returns (result handle, latency in microseconds)."""
    out = C.c_void_p()
    lat = C.c_double()
    _check(lib.cq_server_wait(srv.ptr, ticket, timeout_us, C.byref(out), C.byref(lat)))
    return Handle(out.value, lib.cq_result_destroy, [srv]), lat.value


def cq_server_stats(srv):
    a, b = C.c_uint64(), C.c_uint64()
    _check(lib.cq_server_stats(srv.ptr, C.byref(a), C.byref(b)))
    return a.value, b.value


def cq_result_wait(res, timeout_us: int = 2**64 - 1) -> int:
    return _check(lib.cq_result_wait(res.ptr, timeout_us))


def cq_result_num_groups(res) -> int:
    n = C.c_uint64()
    _check(lib.cq_result_num_groups(res.ptr, C.byref(n)))
    return n.value


def cq_result_fetch(res, out_col: int, n_groups: Optional[int] = None) -> np.ndarray:
    if n_groups is None:
        n_groups = cq_result_num_groups(res)
    kind = C.c_uint32()
    _check(lib.cq_result_column_kind(res.ptr, out_col, C.byref(kind)))
    dt = {0: np.int64, 1: np.uint64, 2: np.float64}[kind.value]
    a = np.empty(n_groups, dtype=dt)
    _check(lib.cq_result_fetch(res.ptr, out_col, a.ctypes.data if n_groups else None, a.nbytes))
    return a


def cq_result_num_columns(res) -> int:
    n = C.c_uint32()
    _check(lib.cq_result_num_columns(res.ptr, C.byref(n)))
    return n.value


def cq_result_key_string(res, key_col: int, row: int) -> bytes:
    s = C.c_char_p()
    n = C.c_uint32()
    _check(lib.cq_result_key_string(res.ptr, key_col, row, C.byref(s), C.byref(n)))
    return C.string_at(s, n.value)


def cq_result_device_time_us(res) -> float:
    t = C.c_double()
    _check(lib.cq_result_device_time_us(res.ptr, C.byref(t)))
    return t.value


def cq_result_kernel_time_us(res) -> float:
    t = C.c_double()
    _check(lib.cq_result_kernel_time_us(res.ptr, C.byref(t)))
    return t.value


def cq_result_device_column(res, out_col: int) -> int:
    p = C.c_void_p()
    _check(lib.cq_result_device_column(res.ptr, out_col, C.byref(p)))
    return p.value


def cq_align_segments(ctx, cols: Sequence[Handle], seg_ends=None, ridx=None, capacity: int = 0, stream=None):
    """Returns the segment count; fills the device buffers when they are given."""
    arr = (C.c_void_p * len(cols))(*[c.ptr for c in cols])
    n = C.c_uint64()
    rc = lib.cq_align_segments(ctx.ptr, C.addressof(arr), len(cols), _stream_ptr(stream),
                               _ptr(seg_ends), _ptr(ridx), capacity, C.byref(n))
    if rc not in (CQ_OK, CQ_ERR_SIZE_MISMATCH) or (rc == CQ_ERR_SIZE_MISMATCH and capacity):
        _check(rc)
    return n.value


def cq_align_segments_static(run_ends, n_rows: int, seg_ends=None, ridx=None, capacity: int = 0, stream=None):
    """Allocation-free alignment over CUDA tensors of run ends (int32 / int64);
    returns the segment count and fills seg_ends / ridx when given."""
    k = len(run_ends)
    ptrs = (C.c_void_p * k)(*[e.data_ptr() for e in run_ends])
    is64 = (C.c_uint32 * k)(*[1 if str(e.dtype).endswith("int64") else 0 for e in run_ends])
    nr = (C.c_uint64 * k)(*[int(e.numel()) for e in run_ends])
    n = C.c_uint64()
    rc = lib.cq_align_segments_static(k, C.addressof(ptrs), C.addressof(is64), C.addressof(nr), int(n_rows),
                                      _stream_ptr(stream), _ptr(seg_ends), _ptr(ridx), capacity, C.byref(n))
    if rc not in (CQ_OK, CQ_ERR_SIZE_MISMATCH) or (rc == CQ_ERR_SIZE_MISMATCH and capacity):
        _check(rc)
    return n.value


# ---------------------------------------------------------------- conveniences
def column_from(ctx, col, device: bool = False) -> Handle:
    """Create a library column from a datagen column (host copy, or borrowed
    CUDA torch tensors when device=True)."""
    if device:
        import torch

        def t(a):
            return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    else:
        def t(a):
            return a
    if col.enc == "rle":
        return cq_column_create_rle(ctx, t(col.run_values), t(col.run_ends), col.n_rows)
    if col.enc == "dict":
        # packed words travel as int32 tensors on the device (same bits)
        return cq_column_create_dict(ctx, col.strings, t(col.words.view(np.int32)) if device else col.words,
                                     col.bit_width, col.n_rows)
    if col.enc == "index":
        return cq_column_create_index(ctx, t(col.values), t(col.positions), col.default, col.n_rows)
    if col.enc == "packed":
        w = t(col.words.view(np.int32)) if device else col.words
        return cq_column_create_bitpacked(ctx, w, col.bit_width, col.base, col.n_rows,
                                          CQ_I64 if col.logical == "i64" else CQ_I32)
    if col.enc == "plain":
        return cq_column_create_plain(ctx, t(col.values))
    if col.enc == "rle_index":   # host arrays only (the library merges them on the host)
        return cq_column_create_rle_index(ctx, col.run_values, col.run_starts, col.run_ends, col.values,
                                          col.positions, col.n_rows)
    raise ValueError(col.enc)


def table_from(ctx, table: dg.Table, device: bool = False):
    cols = [column_from(ctx, c, device) for c in table.columns]
    return cq_table_bind(ctx, cols), cols


def fetch_all(res) -> List[np.ndarray]:
    cq_result_wait(res)
    n = cq_result_num_groups(res)
    return [cq_result_fetch(res, i, n) for i in range(cq_result_num_columns(res))]
