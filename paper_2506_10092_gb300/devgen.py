"""Binding of libcqgen.so, the device-side generator of the nested table's
per-row columns (input infrastructure: it draws and packs values, nothing
else).  The values equal datagen.nested_codes4 / datagen.nested_row_values
row for row; the run-length columns come from datagen.nested_runs."""
from __future__ import annotations

import ctypes as C
import os
from . import datagen as dg

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.path.join(_HERE, "libcqgen.so")
        if not os.path.exists(path):
            raise RuntimeError("libcqgen.so is not built (run paper_2506_10092_gb300.build)")
        _lib = C.CDLL(path)
        _lib.cqgen_hash_fields.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64,
                                           C.c_uint32, C.c_void_p]
        _lib.cqgen_nested_codes4.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64, C.c_uint64,
                                             C.c_uint64, C.c_void_p]
        _lib.cqgen_hash_fields.restype = C.c_int
        _lib.cqgen_nested_codes4.restype = C.c_int
    return _lib


def _words(n_rows: int, bit_width: int):
    import torch
    return torch.empty(dg.padded_word_count(n_rows, bit_width), dtype=torch.int32, device="cuda")


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def hash_fields(n_rows: int, bit_width: int, seed: int, col: int):
    """Device words of the packed fields h(seed, col, r) mod 2^bit_width."""
    w = _words(n_rows, bit_width)
    rc = lib().cqgen_hash_fields(w.data_ptr(), w.numel(), n_rows, bit_width, seed & (2**64 - 1), col, _stream())
    if rc != 0:
        raise RuntimeError(f"cqgen_hash_fields failed ({rc})")
    return w


def nested_codes4(c3_ends_dev, n_rows: int, seed: int):
    """Device words of the nested table's 4-bit c4 codes; c3_ends_dev is the
    c3 run-end array as an int64 CUDA tensor."""
    import torch
    assert c3_ends_dev.dtype == torch.int64 and c3_ends_dev.is_cuda
    w = _words(n_rows, 4)
    rc = lib().cqgen_nested_codes4(w.data_ptr(), w.numel(), c3_ends_dev.data_ptr(), c3_ends_dev.numel(),
                                   n_rows, seed & (2**64 - 1), _stream())
    if rc != 0:
        raise RuntimeError(f"cqgen_nested_codes4 failed ({rc})")
    return w


class DeviceNested:
    """The nested table (lean layout: c1, c2, c3, c4, c7, c8) with its RLE
    columns drawn on the host and its per-row columns generated on the device;
    cq column handles borrow the device buffers held here."""

    def __init__(self, cq, ctx, n_rows: int, seed: int = dg.DEFAULT_SEED, runs=None):
        import torch
        self.n_rows, self.seed = n_rows, seed
        self.runs = runs if runs is not None else dg.nested_runs(n_rows, seed)
        self.dev = []
        handles = []
        for c in self.runs:
            v = torch.from_numpy(c.run_values).cuda()
            e = torch.from_numpy(c.run_ends).cuda()
            self.dev += [v, e]
            handles.append(cq.cq_column_create_rle(ctx, v, e, n_rows))
        e3 = self.dev[-1] if self.dev[-1].dtype == torch.int64 else self.dev[-1].to(torch.int64)
        w4 = nested_codes4(e3, n_rows, seed)
        w7 = hash_fields(n_rows, 8, seed, 7)
        w8 = hash_fields(n_rows, 12, seed, 8)
        self.dev += [e3, w4, w7, w8]
        handles.append(cq.cq_column_create_dict(ctx, dg.NESTED_DICT4, w4, 4, n_rows))
        handles.append(cq.cq_column_create_bitpacked(ctx, w7, 8, dg.NESTED_BASE7, n_rows, cq.CQ_I64))
        handles.append(cq.cq_column_create_bitpacked(ctx, w8, 12, dg.NESTED_BASE8, n_rows, cq.CQ_I64))
        self.columns = handles
        self.table = cq.cq_table_bind(ctx, handles)

    def query_bytes(self, plan) -> int:
        """Compressed bytes a plan over this table reads (its columns)."""
        total = 0
        for c in dg.plan_columns(plan):
            if c < 3:
                total += self.runs[c].run_values.nbytes + self.runs[c].run_ends.nbytes
            else:
                total += (self.n_rows * {3: 4, 4: 8, 5: 12}[c] + 7) // 8
        return total

    def host_table(self) -> dg.Table:
        """The same table on the host (all rows; for tests at small sizes)."""
        import numpy as np
        n = self.n_rows
        r = np.arange(n, dtype=np.int64)
        c1, c2, c3 = self.runs
        c4 = dg.make_dict(dg.NESTED_DICT4, dg.nested_codes4_all(self.seed, c3.run_ends, n), 4)
        c7 = dg.make_packed(dg.nested_row_values(self.seed, 7, r), 8, dg.NESTED_BASE7, "i64")
        c8 = dg.make_packed(dg.nested_row_values(self.seed, 8, r), 12, dg.NESTED_BASE8, "i64")
        return dg.Table([c1, c2, c3, c4, c7, c8], n, ["c1", "c2", "c3", "c4", "c7", "c8"])
