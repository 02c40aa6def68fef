"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It marshals the neutral table / plan
objects of ``paper_2506_10092_gb300.datagen`` into the oracle's own structs;
it never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Dict as TDict, List, Optional

import numpy as np

from . import build as _build

ORC_RLE, ORC_DICT, ORC_INDEX, ORC_PACKED, ORC_PLAIN, ORC_RLE_INDEX, ORC_PACKED_INDEX = 1, 2, 3, 4, 5, 6, 7
_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7}
_AGGS = {"sum": 0, "count": 1, "min": 2, "max": 3, "avg": 4, "var_pop": 5, "var_samp": 6, "std_pop": 7,
         "std_samp": 8}
_FLOAT_AGGS = ("avg", "var_pop", "var_samp", "std_pop", "std_samp")
ORC_ERR_OVERFLOW = -6


class _Col(C.Structure):
    _fields_ = [
        ("enc", C.c_int32), ("n_rows", C.c_uint64),
        ("run_values", C.c_void_p), ("run_ends", C.c_void_p), ("n_runs", C.c_uint64),
        ("words", C.c_void_p), ("n_words", C.c_uint64), ("bit_width", C.c_uint32), ("base", C.c_int64),
        ("idx_values", C.c_void_p), ("positions", C.c_void_p), ("nnz", C.c_uint64), ("default_value", C.c_int64),
        ("values", C.c_void_p),
        ("dict_bytes", C.c_void_p), ("dict_offsets", C.c_void_p), ("n_entries", C.c_uint32),
        ("run_starts", C.c_void_p),
    ]


class _Pred(C.Structure):
    _fields_ = [
        ("col", C.c_uint32), ("op", C.c_int32), ("lo", C.c_int64), ("hi", C.c_int64),
        ("in_ints", C.c_void_p), ("n_in", C.c_uint32),
        ("strs", C.c_void_p), ("str_lens", C.c_void_p), ("n_strs", C.c_uint32),
        ("or_group", C.c_uint32), ("negate", C.c_uint32),
    ]


class _Node(C.Structure):
    _fields_ = [("kind", C.c_int32), ("arg", C.c_uint32)]


_NODES = {"pred": 0, "and": 1, "or": 2, "not": 3}


class _Agg(C.Structure):
    _fields_ = [("op", C.c_int32), ("col", C.c_uint32), ("expr", C.c_int32), ("col2", C.c_uint32)]


_EXPRS = {None: 0, "add": 1, "sub": 2, "mul": 3}


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.orc_decode.argtypes = [C.POINTER(_Col), C.c_uint64, C.c_uint64, C.c_void_p]
            L.orc_query.argtypes = [C.POINTER(_Col), C.c_uint32, C.c_uint64, C.POINTER(_Pred), C.c_uint32,
                                    C.POINTER(_Node), C.c_uint32, C.c_void_p, C.c_uint32, C.POINTER(_Agg), C.c_uint32,
                                    C.c_void_p, C.c_uint32, C.c_uint32, C.POINTER(C.c_void_p)]
            L.orc_result_status.argtypes = [C.c_void_p]
            L.orc_result_num_groups.argtypes = [C.c_void_p]
            L.orc_result_num_groups.restype = C.c_uint64
            L.orc_result_keys.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p]
            L.orc_result_agg.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p]
            L.orc_result_sum128.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]
            L.orc_result_free.argtypes = [C.c_void_p]
            L.orc_div_round.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_div_round.restype = C.c_double
            L.orc_align.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.c_uint64,
                                    C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p]
            L.orc_join_index.argtypes = [C.POINTER(_Col), C.POINTER(_Col), C.POINTER(C.c_uint64), C.c_void_p,
                                         C.c_void_p]
            L.orc_apply_join_index.argtypes = [C.POINTER(_Col), C.c_void_p, C.c_uint64, C.c_void_p]
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


class _Marshal:
    """Keeps every buffer handed to the oracle alive for the call."""

    def __init__(self):
        self.keep = []

    def k(self, a):
        self.keep.append(a)
        return a

    def column(self, c) -> _Col:
        s = _Col()
        s.enc = {"rle": ORC_RLE, "dict": ORC_DICT, "index": ORC_INDEX, "packed": ORC_PACKED, "plain": ORC_PLAIN,
                 "rle_index": ORC_RLE_INDEX, "packed_index": ORC_PACKED_INDEX}[c.enc]
        s.n_rows = int(c.n_rows)
        if c.enc == "rle":
            v, e = self.k(_i64(c.run_values)), self.k(_i64(c.run_ends))
            s.run_values, s.run_ends, s.n_runs = _p(v), _p(e), int(e.shape[0])
        elif c.enc in ("packed", "dict"):
            w = self.k(np.ascontiguousarray(c.words, dtype=np.uint32))
            s.words, s.n_words, s.bit_width = _p(w), int(w.shape[0]), int(c.bit_width)
            if c.enc == "packed":
                s.base = int(c.base)
            else:
                b = self.k(np.ascontiguousarray(c.dict_bytes, dtype=np.uint8))
                o = self.k(np.ascontiguousarray(c.dict_offsets, dtype=np.uint64))
                s.dict_bytes, s.dict_offsets, s.n_entries = _p(b), o.ctypes.data, len(c.strings)
        elif c.enc == "index":
            v, p = self.k(_i64(c.values)), self.k(_i64(c.positions))
            s.idx_values, s.positions, s.nnz, s.default_value = _p(v), _p(p), int(p.shape[0]), int(c.default)
        elif c.enc == "plain":
            v = self.k(_i64(c.values))
            s.values = _p(v)
        elif c.enc == "packed_index":
            w = self.k(np.ascontiguousarray(c.words, dtype=np.uint32))
            s.words, s.n_words, s.bit_width, s.base = _p(w), int(w.shape[0]), int(c.bit_width), int(c.base)
            v, p = self.k(_i64(c.values)), self.k(_i64(c.positions))
            s.idx_values, s.positions, s.nnz = _p(v), _p(p), int(p.shape[0])
        elif c.enc == "rle_index":
            rv, rs, re_ = self.k(_i64(c.run_values)), self.k(_i64(c.run_starts)), self.k(_i64(c.run_ends))
            s.run_values, s.run_starts, s.run_ends, s.n_runs = _p(rv), _p(rs), _p(re_), int(rs.shape[0])
            v, p = self.k(_i64(c.values)), self.k(_i64(c.positions))
            s.idx_values, s.positions, s.nnz = _p(v), _p(p), int(p.shape[0])
        return s

    def pred(self, p) -> _Pred:
        s = _Pred()
        s.col, s.op, s.lo, s.hi = int(p.col), _OPS[p.op], int(p.lo), int(p.hi)
        s.or_group, s.negate = int(getattr(p, "group", 0)), 1 if getattr(p, "neg", False) else 0
        if p.ints is not None:
            a = self.k(_i64(list(p.ints)))
            s.in_ints, s.n_in = _p(a), int(a.shape[0])
        if p.strs is not None:
            bufs = [self.k(C.create_string_buffer(bytes(x), len(x) + 1)) for x in p.strs]
            ptrs = self.k((C.c_void_p * max(1, len(bufs)))(*[C.addressof(b) for b in bufs]))
            lens = self.k(np.array([len(x) for x in p.strs] or [0], dtype=np.uint32))
            s.strs, s.str_lens, s.n_strs = C.addressof(ptrs), lens.ctypes.data, len(bufs)
        return s


@dataclass
class OracleResult:
    status: int
    keys: List[np.ndarray]           # one int64 array per group-by column
    aggs: List[np.ndarray]           # int64 (SUM/MIN/MAX), uint64 (COUNT), float64 (AVG/VAR/STD)
    sum128: TDict[int, tuple]        # agg index -> (lo uint64[], hi int64[]) for SUM/AVG

    @property
    def num_groups(self) -> int:
        return int(self.keys[0].shape[0]) if self.keys else (int(self.aggs[0].shape[0]) if self.aggs else 1)


def query(table, plan, row_ranges=None, n_threads: int = 1) -> OracleResult:
    L = lib()
    m = _Marshal()
    cols = (_Col * len(table.columns))(*[m.column(c) for c in table.columns])
    preds = (_Pred * max(1, len(plan.preds)))(*[m.pred(p) for p in plan.preds])
    aggs = (_Agg * max(1, len(plan.aggs)))(*[_Agg(_AGGS[a.op], int(a.col), _EXPRS[getattr(a, "expr", None)],
                                                   int(getattr(a, "col2", 0))) for a in plan.aggs])
    prog = list(getattr(plan, "filter", None) or [])
    nodes = (_Node * max(1, len(prog)))(*[_Node(_NODES[k], int(a)) for k, a in prog])
    gb = m.k(np.array(list(plan.group_by) or [0], dtype=np.uint32))
    rr = None
    nr = 0
    if row_ranges is not None:
        rr = m.k(np.ascontiguousarray(np.asarray(row_ranges, dtype=np.uint64).reshape(-1)))
        nr = rr.shape[0] // 2
    out = C.c_void_p()
    rc = L.orc_query(cols, len(table.columns), int(table.n_rows), preds, len(plan.preds), nodes, len(prog),
                     gb.ctypes.data, len(plan.group_by), aggs, len(plan.aggs),
                     None if rr is None else rr.ctypes.data, nr, int(n_threads), C.byref(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the query (status {rc})")
    try:
        g = int(L.orc_result_num_groups(out))
        status = int(L.orc_result_status(out))
        keys = []
        for k in range(len(plan.group_by)):
            a = np.empty(g, dtype=np.int64)
            L.orc_result_keys(out, k, a.ctypes.data)
            keys.append(a)
        res_aggs = []
        s128 = {}
        for i, a in enumerate(plan.aggs):
            dt = np.uint64 if a.op == "count" else (np.float64 if a.op in _FLOAT_AGGS else np.int64)
            x = np.empty(g, dtype=dt)
            L.orc_result_agg(out, i, x.ctypes.data)
            res_aggs.append(x)
            if a.op in ("sum", "avg"):
                lo = np.empty(g, dtype=np.uint64)
                hi = np.empty(g, dtype=np.int64)
                L.orc_result_sum128(out, i, lo.ctypes.data, hi.ctypes.data)
                s128[i] = (lo, hi)
        return OracleResult(status, keys, res_aggs, s128)
    finally:
        L.orc_result_free(out)


def decode(col, row_begin: int = 0, row_end: Optional[int] = None) -> np.ndarray:
    L = lib()
    m = _Marshal()
    s = m.column(col)
    if row_end is None:
        row_end = int(col.n_rows)
    out = np.empty(max(0, row_end - row_begin), dtype=np.int64)
    rc = L.orc_decode(C.byref(s), int(row_begin), int(row_end), out.ctypes.data if out.size else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the column (status {rc})")
    return out


def align(run_ends_list, n_rows: int):
    """(segment ends int64[S], run indices int64[k, S]) of the common refinement."""
    L = lib()
    ends = [_i64(e) for e in run_ends_list]
    k = len(ends)
    ptrs = (C.c_void_p * max(1, k))(*[e.ctypes.data if e.size else None for e in ends])
    nr = np.array([e.shape[0] for e in ends] or [0], dtype=np.uint64)
    ns = C.c_uint64()
    rc = L.orc_align(k, C.addressof(ptrs), nr.ctypes.data, int(n_rows), C.byref(ns), None, None)
    if rc != 0:
        raise ValueError(f"oracle rejected the run ends (status {rc})")
    S = int(ns.value)
    seg = np.empty(S, dtype=np.int64)
    ridx = np.empty((k, S), dtype=np.int64)
    L.orc_align(k, C.addressof(ptrs), nr.ctypes.data, int(n_rows), C.byref(ns),
                seg.ctypes.data if S else None, ridx.ctypes.data if S * k else None)
    return seg, ridx


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def div_round(n: int, d: int) -> float:
    """The oracle's correctly rounded n / d (0 <= n < 2^256, 0 < d < 2^128)."""
    L = lib()
    nn = np.array([(n >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    dd = np.array([(d >> (64 * i)) & (2**64 - 1) for i in range(2)], dtype=np.uint64)
    return float(L.orc_div_round(nn.ctypes.data, dd.ctypes.data))


def join_index(left, right):
    """(left rows, right rows) of every pair with equal values, ascending."""
    L = lib()
    m = _Marshal()
    a, b = m.column(left), m.column(right)
    n = C.c_uint64()
    rc = L.orc_join_index(C.byref(a), C.byref(b), C.byref(n), None, None)
    if rc != 0:
        raise ValueError(f"oracle rejected the join (status {rc})")
    li = np.empty(int(n.value), dtype=np.int64)
    ri = np.empty(int(n.value), dtype=np.int64)
    if n.value:
        L.orc_join_index(C.byref(a), C.byref(b), C.byref(n), li.ctypes.data, ri.ctypes.data)
    return li, ri


def apply_join_index(col, rows):
    L = lib()
    m = _Marshal()
    s = m.column(col)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(r.shape[0], dtype=np.int64)
    rc = L.orc_apply_join_index(C.byref(s), r.ctypes.data if r.size else None, int(r.shape[0]),
                                out.ctypes.data if out.size else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the rows (status {rc})")
    return out
