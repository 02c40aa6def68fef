"""Seeded synthetic tables of lightweight-compressed columns.

This module only *draws* values and *encodes* them (run-length, dictionary,
sparse index with a default, bit packing).  It holds none of the query
arithmetic: nothing here filters, aligns, groups or aggregates.  Both the CPU
oracle (tests only) and the CUDA library consume the objects built here, so
the same seeded input reaches both sides.

Encodings follow the tensor representations of Section 3 of the paper
(Plain, RLE, Index, dictionary codes, bit-width reduction):

* ``RLE``     run values + *exclusive* run ends (row ``r`` belongs to run ``i``
              iff ``ends[i-1] <= r < ends[i]``); the paper's inclusive
              ``start..end`` form is ``start = ends[i-1]``, ``end = ends[i]-1``.
* ``Index``   sorted unique positions + values; every unlisted row holds
              ``default``.
* ``Dict``    a bytewise-sorted unique dictionary of strings plus per-row codes
              bit-packed LSB-first into little-endian uint32 words.
* ``Packed``  per-row unsigned offsets bit-packed like ``Dict`` codes; the
              logical value is ``base + offset`` (frame of reference).
* ``Plain``   one value per row.

Packed word buffers are padded to a 16-byte multiple plus one extra 16-byte
vector, which is the padding the C-ABI asks of borrowed device buffers.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

DEFAULT_SEED = 20250611


# --------------------------------------------------------------------------
# column containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class RLE:
    run_values: np.ndarray          # int32 or int64, [R]
    run_ends: np.ndarray            # int32 or int64, [R], strictly increasing, last == n_rows
    n_rows: int
    enc: str = "rle"


@dataclasses.dataclass
class Index:
    values: np.ndarray              # int32 or int64, [nnz]
    positions: np.ndarray           # int32 or int64, [nnz], sorted unique, < n_rows
    default: int
    n_rows: int
    enc: str = "index"


@dataclasses.dataclass
class Dict:
    strings: List[bytes]            # sorted bytewise, unique
    words: np.ndarray               # uint32 packed codes
    bit_width: int
    n_rows: int
    enc: str = "dict"

    @property
    def dict_bytes(self) -> np.ndarray:
        return np.frombuffer(b"".join(self.strings), dtype=np.uint8).copy()

    @property
    def dict_offsets(self) -> np.ndarray:
        lens = np.array([len(s) for s in self.strings], dtype=np.uint64)
        off = np.zeros(len(self.strings) + 1, dtype=np.uint64)
        np.cumsum(lens, out=off[1:])
        return off


@dataclasses.dataclass
class Packed:
    words: np.ndarray               # uint32 packed offsets
    bit_width: int
    base: int
    n_rows: int
    logical: str = "i64"            # "i32" or "i64"
    enc: str = "packed"


@dataclasses.dataclass
class Plain:
    values: np.ndarray              # int32 or int64, [n_rows]
    enc: str = "plain"

    @property
    def n_rows(self) -> int:
        return int(self.values.shape[0])


@dataclasses.dataclass
class Table:
    columns: list
    n_rows: int
    names: Optional[List[str]] = None


# --------------------------------------------------------------------------
# query plans (a neutral description both sides translate)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Pred:
    col: int
    op: str                         # lt le gt ge eq ne between in
    lo: int = 0
    hi: int = 0
    ints: Optional[Sequence[int]] = None      # IN list on integer columns
    strs: Optional[Sequence[bytes]] = None    # literals on dictionary columns


@dataclasses.dataclass
class Agg:
    op: str                         # sum count min max avg
    col: int = 0                    # ignored for count


@dataclasses.dataclass
class Plan:
    preds: List[Pred]
    group_by: List[int]
    aggs: List[Agg]


# --------------------------------------------------------------------------
# encoders (offline conversion, Section 2.1 / Table 1 plain_to_rle)
# --------------------------------------------------------------------------
def padded_word_count(n_rows: int, bit_width: int) -> int:
    """uint32 words for n_rows fields of bit_width bits, rounded up to a
    16-byte multiple plus one extra 16-byte vector."""
    need = (n_rows * bit_width + 31) // 32
    return ((need + 3) // 4) * 4 + 4


def pack_bits(offsets: np.ndarray, bit_width: int) -> np.ndarray:
    """Pack unsigned fields LSB-first: field i occupies stream bits
    [i*w, (i+1)*w) and stream bit b is bit (b % 32) of word b // 32."""
    w = int(bit_width)
    if not 1 <= w <= 64:
        raise ValueError("bit width must be in 1..64")
    offsets = np.asarray(offsets)
    n = int(offsets.shape[0])
    out = np.zeros(padded_word_count(n, w), dtype=np.uint32)
    if n == 0:
        return out
    u = offsets.astype(np.uint64, copy=False)
    if w < 64 and np.any(u >> np.uint64(w)):
        raise ValueError("offset does not fit the bit width")
    # G consecutive fields fill exactly W whole words (G*w == 32*W)
    g = int(np.gcd(w, 32))
    G, W = 32 // g, w // g
    n_groups = (n + G - 1) // G
    v = np.zeros(n_groups * G, dtype=np.uint64)
    v[:n] = u
    v = v.reshape(n_groups, G)
    words = np.zeros((n_groups, W + 2), dtype=np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    for j in range(G):
        bit = j * w
        q, s = bit // 32, bit % 32
        f = v[:, j]
        words[:, q] |= (f << np.uint64(s)) & m32
        if s + w > 32:
            words[:, q + 1] |= (f >> np.uint64(32 - s)) & m32
        if s + w > 64:
            words[:, q + 2] |= (f >> np.uint64(64 - s)) & m32
    flat = words[:, :W].astype(np.uint32).reshape(-1)
    need = (n * w + 31) // 32
    out[:need] = flat[:need]
    return out


def rle_encode(values: np.ndarray, end_dtype=None):
    """Maximal runs of a plain array (plain_to_rle of Table 1)."""
    values = np.asarray(values)
    n = values.shape[0]
    if n == 0:
        return values[:0].copy(), np.zeros(0, dtype=end_dtype or np.int64)
    change = np.flatnonzero(values[1:] != values[:-1]) + 1
    ends = np.concatenate([change, [n]])
    vals = values[ends - 1]
    if end_dtype is None:
        end_dtype = np.int32 if n < 2**31 else np.int64
    return vals.copy(), ends.astype(end_dtype)


def geometric_ends(rng: np.random.Generator, n_rows: int, mean: float, end_dtype=None) -> np.ndarray:
    """Exclusive run ends with run lengths ~ Geometric(p = 1/mean) on {1,2,...};
    the last run is truncated so the lengths sum to n_rows exactly."""
    if end_dtype is None:
        end_dtype = np.int32 if n_rows < 2**31 else np.int64
    if n_rows == 0:
        return np.zeros(0, dtype=end_dtype)
    p = min(1.0, 1.0 / float(mean))
    parts = []
    total = 0
    while total < n_rows:
        k = int((n_rows - total) / mean * 1.05) + 64
        lens = rng.geometric(p, size=k).astype(np.int64)
        parts.append(lens)
        total += int(lens.sum())
    lens = np.concatenate(parts)
    ends = np.cumsum(lens)
    r = int(np.searchsorted(ends, n_rows, side="left")) + 1
    ends = ends[:r]
    ends[-1] = n_rows
    return ends.astype(end_dtype)


def random_strings(rng: np.random.Generator, n: int, min_len: int, max_len: int) -> List[bytes]:
    """n unique random strings over [A-Za-z0-9], sorted bytewise."""
    alphabet = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789", dtype=np.uint8)
    out = set()
    while len(out) < n:
        need = n - len(out)
        lens = rng.integers(min_len, max_len + 1, size=need)
        chars = alphabet[rng.integers(0, alphabet.shape[0], size=int(lens.sum()))]
        pos = 0
        for L in lens:
            out.add(chars[pos:pos + L].tobytes())
            pos += L
    return sorted(out)


def zipf_ranks(rng: np.random.Generator, n: int, n_ranks: int, s: float, chunk: int = 1 << 24) -> np.ndarray:
    """Draw n ranks in 0..n_ranks-1 with P(rank k) proportional to (k+1)^-s
    (inverse CDF of a uniform draw; a guide table resolves most draws)."""
    p = np.arange(1, n_ranks + 1, dtype=np.float64) ** (-float(s))
    cum = np.cumsum(p)
    cum /= cum[-1]
    B = 1 << 20
    edges = np.arange(B + 1, dtype=np.float64) / B
    guide = np.searchsorted(cum, edges, side="right")
    np.minimum(guide, n_ranks - 1, out=guide)
    lo, hi = guide[:-1], guide[1:]
    out = np.empty(n, dtype=np.int32)
    for c0 in range(0, n, chunk):
        u = rng.random(min(chunk, n - c0))
        b = (u * B).astype(np.int64)
        r = lo[b].copy()
        amb = np.flatnonzero(lo[b] != hi[b])
        if amb.shape[0]:
            r[amb] = np.minimum(np.searchsorted(cum, u[amb], side="right"), n_ranks - 1)
        out[c0:c0 + u.shape[0]] = r
    return out


# --------------------------------------------------------------------------
# column builders
# --------------------------------------------------------------------------
def make_rle(rng, n_rows, mean_run, lo, hi, val_dtype=np.int32, end_dtype=None) -> RLE:
    ends = geometric_ends(rng, n_rows, mean_run, end_dtype)
    vals = rng.integers(lo, hi + 1, size=ends.shape[0], dtype=np.int64).astype(val_dtype)
    return RLE(vals, ends, n_rows)


def make_packed(offsets: np.ndarray, bit_width: int, base: int, logical: str = "i64") -> Packed:
    return Packed(pack_bits(offsets, bit_width), bit_width, int(base), int(offsets.shape[0]), logical)


def make_dict(strings: List[bytes], codes: np.ndarray, bit_width: int) -> Dict:
    return Dict(list(strings), pack_bits(codes, bit_width), bit_width, int(codes.shape[0]))


def make_index(rng, n_rows, nnz, lo, hi, default=0, val_dtype=np.int64, pos_dtype=None) -> Index:
    if pos_dtype is None:
        pos_dtype = np.int32 if n_rows < 2**31 else np.int64
    pos = np.sort(rng.choice(n_rows, size=nnz, replace=False)).astype(pos_dtype) if nnz else np.zeros(0, pos_dtype)
    vals = rng.integers(lo, hi + 1, size=nnz, dtype=np.int64).astype(val_dtype)
    return Index(vals, pos, int(default), n_rows)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def tiny_two_rle(n_rows: int = 1_000_000, seed: int = DEFAULT_SEED):
    """Two int32 RLE columns.  A: geometric runs (mean 8), values U{0..99};
    B: geometric runs (mean 5), values U{0..9}.
    Query: SELECT B, SUM(A), COUNT(*) WHERE A < 50 GROUP BY B."""
    rng = np.random.default_rng([seed, 1])
    a = make_rle(rng, n_rows, 8.0, 0, 99)
    b = make_rle(rng, n_rows, 5.0, 0, 9)
    table = Table([a, b], n_rows, ["A", "B"])
    plan = Plan([Pred(0, "lt", 50)], [1], [Agg("sum", 0), Agg("count")])
    return table, plan


def heterogeneous(n_rows: int = 100_000_000, seed: int = DEFAULT_SEED, n_in: int = 64,
                  index_default: int = 0, nnz: Optional[int] = None):
    """Five columns in four encodings.
    c1 int32 RLE key, geometric runs mean 1000, values U{0..999};
    c2 dictionary of 10,000 strings (8-24 chars of [A-Za-z0-9]) with Zipf(1.1)
       frequencies through a seeded rank->code permutation, 14-bit packed codes;
    c3 int64 index-encoded, 1% of rows listed (sorted int32 positions),
       values U[-2^40, 2^40], default ``index_default``;
    c4 plain int32 U{0..1,000,000};
    c5 int64 bit-width reduced: base 2^32+12345 plus a 20-bit offset.
    Query: SELECT c1, c2, SUM(c3), SUM(c5), MIN(c5), MAX(c5), COUNT(*)
           WHERE c2 IN (n_in strings: 8 of the 20 most frequent + the rest
           uniform) AND c4 BETWEEN 250000 AND 749999 GROUP BY c1, c2."""
    rng = np.random.default_rng([seed, 2])
    n_dict = 10_000
    c1 = make_rle(rng, n_rows, 1000.0, 0, 999)
    strings = random_strings(rng, n_dict, 8, 24)
    perm = rng.permutation(n_dict)                     # rank -> code
    ranks = zipf_ranks(rng, n_rows, n_dict, 1.1)
    codes = perm[ranks].astype(np.uint32)
    del ranks
    c2 = make_dict(strings, codes, 14)
    del codes
    if nnz is None:
        nnz = n_rows // 100
    c3 = make_index(rng, n_rows, nnz, -(1 << 40), 1 << 40, default=index_default)
    c4 = Plain(rng.integers(0, 1_000_001, size=n_rows, dtype=np.int32))
    off5 = rng.integers(0, 1 << 20, size=n_rows, dtype=np.uint32)
    c5 = make_packed(off5, 20, (1 << 32) + 12345, "i64")
    del off5
    hot = rng.choice(20, size=min(8, n_in), replace=False)
    rest_pool = np.arange(20, n_dict)
    rest = rng.choice(rest_pool, size=max(0, n_in - hot.shape[0]), replace=False)
    in_codes = perm[np.concatenate([hot, rest])]
    in_strs = [strings[int(c)] for c in in_codes]
    table = Table([c1, c2, c3, c4, c5], n_rows, ["c1", "c2", "c3", "c4", "c5"])
    plan = Plan(
        [Pred(1, "in", strs=in_strs), Pred(3, "between", 250_000, 749_999)],
        [0, 1],
        [Agg("sum", 2), Agg("sum", 4), Agg("min", 4), Agg("max", 4), Agg("count")],
    )
    return table, plan


def compressed_bytes(table: Table, cols: Optional[Sequence[int]] = None) -> int:
    """Bytes the method must read for the listed columns (all by default):
    RLE R*(value+end), packed/dict N*w/8, index nnz*(position+value),
    plain N*element size.  Dictionary strings are not counted."""
    total = 0
    idx = range(len(table.columns)) if cols is None else cols
    for i in idx:
        c = table.columns[i]
        if c.enc == "rle":
            total += c.run_values.nbytes + c.run_ends.nbytes
        elif c.enc in ("dict", "packed"):
            total += (c.n_rows * c.bit_width + 7) // 8
        elif c.enc == "index":
            total += c.values.nbytes + c.positions.nbytes
        elif c.enc == "plain":
            total += c.values.nbytes
    return total


def plan_columns(plan: Plan) -> List[int]:
    cols = set()
    for p in plan.preds:
        cols.add(p.col)
    cols.update(plan.group_by)
    for a in plan.aggs:
        if a.op != "count":
            cols.add(a.col)
    return sorted(cols)
