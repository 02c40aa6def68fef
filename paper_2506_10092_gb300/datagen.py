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
from typing import List, Optional, Sequence, Tuple

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
class RLEIndex:
    """RLE + Index composite (Section 3.2): runs [run_starts[i], run_ends[i])
    hold run_values[i]; rows positions[k] hold values[k]; together they cover
    every row exactly once."""
    run_values: np.ndarray          # [R]
    run_starts: np.ndarray          # [R], sorted
    run_ends: np.ndarray            # [R], exclusive
    values: np.ndarray              # [nnz]
    positions: np.ndarray           # [nnz], sorted unique
    n_rows: int
    enc: str = "rle_index"


@dataclasses.dataclass
class PackedIndex:
    """Plain + Index composite (Section 3.2, outlier patching): a narrow
    bit-packed field per row (base + field) and the outliers listed by
    position; the fields at listed rows hold anything and are never read."""
    words: np.ndarray               # uint32 packed fields
    bit_width: int
    base: int
    values: np.ndarray              # [nnz] outliers
    positions: np.ndarray           # [nnz], sorted unique
    n_rows: int
    enc: str = "packed_index"


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
    group: int = 0                  # 0: a conjunct of its own; g > 0: OR-ed with group g's others
    neg: bool = False               # the predicate's complement (NOT)


@dataclasses.dataclass
class Agg:
    op: str                         # sum count min max avg var_pop var_samp std_pop std_samp
    col: int = 0                    # ignored for count
    expr: Optional[str] = None      # "add" / "sub" / "mul": the input is col (expr) col2, row by row
    col2: int = 0


@dataclasses.dataclass
class Plan:
    preds: List[Pred]
    group_by: List[int]
    aggs: List[Agg]
    # optional boolean filter over the predicates, postfix: ("pred", i),
    # ("and", k), ("or", k) (pop k >= 1 values), ("not", 0); None = the AND
    # of the conjuncts
    filter: Optional[List[Tuple[str, int]]] = None


FILTER_NODES = {"pred": 0, "and": 1, "or": 2, "not": 3}


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
def rle_index_encode(values: np.ndarray, min_run: int) -> RLEIndex:
    """RLE + Index of a value sequence: runs of equal values at least
    min_run long are RLE runs, the rows of shorter runs are index entries."""
    v = np.asarray(values, dtype=np.int64)
    n = int(v.shape[0])
    if n == 0:
        z = np.zeros(0, np.int64)
        return RLEIndex(z, z, z, z, z, 0)
    brk = np.flatnonzero(v[1:] != v[:-1]) + 1
    starts = np.concatenate([[0], brk]).astype(np.int64)
    ends = np.concatenate([brk, [n]]).astype(np.int64)
    long_ = (ends - starts) >= min_run
    pos = np.concatenate([np.arange(s, e, dtype=np.int64) for s, e in zip(starts[~long_], ends[~long_])]) \
        if (~long_).any() else np.zeros(0, np.int64)
    return RLEIndex(v[starts[long_]], starts[long_], ends[long_], v[pos], pos, n)


def packed_index_encode(values: np.ndarray, bit_width: int, fill: Optional[np.ndarray] = None) -> PackedIndex:
    """Plain + Index of a value sequence: the values in [base, base +
    2^bit_width) around the median (centering) are packed, the rest listed;
    the packed fields at listed rows take `fill` (default 0)."""
    v = np.asarray(values, dtype=np.int64)
    n = int(v.shape[0])
    base = int(np.median(v)) - (1 << (bit_width - 1)) if n else 0
    off = v.astype(object) - base
    inl = np.array([0 <= int(x) < (1 << bit_width) for x in off], dtype=bool)
    pos = np.flatnonzero(~inl).astype(np.int64)
    fields = np.where(inl, off, 0).astype(np.uint64) if n else np.zeros(0, np.uint64)
    if fill is not None and pos.size:
        fields[pos] = np.asarray(fill, dtype=np.uint64)[:pos.size] & np.uint64((1 << bit_width) - 1)
    return PackedIndex(pack_bits(fields, bit_width), bit_width, base, v[pos], pos, n)


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
def tiny_two_rle(n_rows: int = 1_000_000, seed: int = DEFAULT_SEED, mean_a: float = 8.0, mean_b: float = 5.0):
    """Two int32 RLE columns.  A: geometric runs (mean 8), values U{0..99};
    B: geometric runs (mean 5), values U{0..9} (other means for run-length
    sweeps).  Query: SELECT B, SUM(A), COUNT(*) WHERE A < 50 GROUP BY B."""
    rng = np.random.default_rng([seed, 1])
    a = make_rle(rng, n_rows, mean_a, 0, 99)
    b = make_rle(rng, n_rows, mean_b, 0, 9)
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


# --------------------------------------------------------------------------
# counter-based per-row values
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, col: int, idx: np.ndarray) -> np.ndarray:
    """h(seed, col, i): the SplitMix64 output function (Steele, Lea and Flood,
    "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
    the counter state (seed XOR col << 56) + (i + 1) * 0x9E3779B97F4A7C15,
    all arithmetic mod 2^64.  A pure function of (seed, col, i), so any row or
    prefix can be produced alone."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(col & 0xFF) << np.uint64(56))) + \
            (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _nested_ends(rng, n_rows: int, mean: float, parent_ends: Optional[np.ndarray], end_dtype) -> np.ndarray:
    """Run ends of a column sorted inside its parent's runs: the parent's ends
    plus geometric(mean) boundaries of its own."""
    own = geometric_ends(rng, n_rows, mean, np.int64)
    if parent_ends is None:
        return own.astype(end_dtype)
    # merge two sorted unique arrays: insert the parent ends the child lacks
    par = parent_ends.astype(np.int64)
    pos = np.searchsorted(own, par, side="left")
    new = (pos >= own.shape[0]) | (own[np.minimum(pos, own.shape[0] - 1)] != par)
    return np.insert(own, pos[new], par[new]).astype(end_dtype)


def _increasing_in_parent(rng, ends: np.ndarray, parent_ends: np.ndarray, domain: int) -> np.ndarray:
    """Run values strictly increasing inside every parent run, in 0..domain-1:
    the j-th of k runs of a parent run takes a seeded value in its own slice
    [floor(j*domain/k), floor((j+1)*domain/k)) (non-decreasing if k > domain)."""
    parent_of = np.searchsorted(parent_ends.astype(np.int64), ends.astype(np.int64), side="left")
    first = np.searchsorted(parent_of, np.arange(parent_ends.shape[0]), side="left")
    k = np.diff(np.concatenate([first, [ends.shape[0]]]))[parent_of]
    j = np.arange(ends.shape[0]) - first[parent_of]
    lo = (j * domain) // k
    hi = ((j + 1) * domain) // k
    width = np.maximum(hi - lo, 1)
    v = lo + rng.integers(0, 1 << 62, size=ends.shape[0]) % width
    return np.minimum(v, domain - 1)


NESTED_BASE7 = (1 << 20) - 3
NESTED_BASE8 = 777_777


def nested_codes4(seed: int, c3_ends: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """c4 of the nested table at the given rows: inside each c3 run of
    length L the code is the number of the run's 15 cut points
    h(seed, 4, 15 * run + k) mod L (k = 0..14) at or before the row's offset
    in the run -- non-decreasing along the run, 0..15."""
    ends = c3_ends.astype(np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    run = np.searchsorted(ends, rows, side="right")
    start = np.where(run > 0, ends[np.maximum(run - 1, 0)], 0)
    length = (ends[run] - start).astype(np.uint64)
    off = (rows - start).astype(np.uint64)
    code = np.zeros(rows.shape[0], dtype=np.uint32)
    base = run.astype(np.uint64) * np.uint64(15)
    for k in range(15):
        cut = splitmix64(seed, 4, base + np.uint64(k)) % length
        code += (off >= cut).astype(np.uint32)
    return code


def nested_codes4_all(seed: int, c3_ends: np.ndarray, n_rows: int) -> np.ndarray:
    """nested_codes4 for every row at once: each cut point adds one at its
    row, and the code is the running count inside the run."""
    ends = c3_ends.astype(np.int64)
    if n_rows == 0:
        return np.zeros(0, np.uint32)
    starts = np.concatenate([[0], ends[:-1]])
    length = (ends - starts).astype(np.uint64)
    base = np.arange(ends.shape[0], dtype=np.uint64) * np.uint64(15)
    inc = np.zeros(n_rows + 1, dtype=np.int32)
    for k in range(15):
        cut = (splitmix64(seed, 4, base + np.uint64(k)) % length).astype(np.int64)
        np.add.at(inc, starts + cut, 1)
    run_total = np.cumsum(inc[:-1], dtype=np.int64)
    before = np.concatenate([[0], run_total])[starts]        # count before each run starts
    return (run_total - np.repeat(before, ends - starts)).astype(np.uint32)


def nested_row_values(seed: int, col: int, rows: np.ndarray) -> np.ndarray:
    """Per-row fields of columns c5..c8 of the nested table (unsigned codes /
    offsets): c5 8 bits, c6 16 bits, c7 8 bits, c8 12 bits of h(seed, col, row)."""
    bits = {5: 8, 6: 16, 7: 8, 8: 12}[col]
    return (splitmix64(seed, col, rows) & np.uint64((1 << bits) - 1)).astype(np.uint32)


def nested(n_rows: int, seed: int = DEFAULT_SEED, lo3: int = 200, hi3: int = 699, lean: bool = False):
    """A lexicographically sorted 8-column table (nested RLE).
    c1 RLE, runs mean 1e6, value = run ordinal;
    c2 RLE inside c1 runs (own boundaries mean 1e4), values strictly
       increasing within each c1 run, 0..9999;
    c3 RLE inside c2 runs (own boundaries mean 1e2), increasing within each
       c2 run, 0..999;
    c4 4-bit dictionary code, non-decreasing within each c3 run (15 seeded
       cut points per run), bit-packed;
    c5 8-bit and c6 16-bit dictionary codes, c7 int64 = 2^20-3 + 8-bit offset,
    c8 int64 = 777777 + 12-bit offset, all per-row counter-based values
       (splitmix64), bit-packed.
    Run ends are int64 when n_rows >= 2^31.  ``lean`` leaves out c5 and c6,
    which the query does not read (column indices then shift; use
    nested_plan(..., lean=True)).
    Query: SELECT c2, c4, SUM(c7), SUM(c8) WHERE c3 BETWEEN lo3 AND hi3
           GROUP BY c2, c4."""
    c1, c2, c3 = nested_runs(n_rows, seed)
    rows = np.arange(n_rows, dtype=np.int64)
    c4 = make_dict(NESTED_DICT4, nested_codes4_all(seed, c3.run_ends, n_rows), 4)
    c7 = make_packed(nested_row_values(seed, 7, rows), 8, NESTED_BASE7, "i64")
    c8 = make_packed(nested_row_values(seed, 8, rows), 12, NESTED_BASE8, "i64")
    if lean:
        table = Table([c1, c2, c3, c4, c7, c8], n_rows, ["c1", "c2", "c3", "c4", "c7", "c8"])
        return table, nested_plan(lo3, hi3, lean=True)
    c5 = make_dict([b"h%03d" % i for i in range(256)], nested_row_values(seed, 5, rows), 8)
    c6 = make_dict([b"w%05d" % i for i in range(1 << 16)], nested_row_values(seed, 6, rows), 16)
    table = Table([c1, c2, c3, c4, c5, c6, c7, c8], n_rows, ["c1", "c2", "c3", "c4", "c5", "c6", "c7", "c8"])
    return table, nested_plan(lo3, hi3)


NESTED_DICT4 = [b"g%02d" % i for i in range(16)]


def nested_runs(n_rows: int, seed: int = DEFAULT_SEED):
    """The three RLE columns c1, c2, c3 of the nested table (see nested);
    drawn on the host, the per-row columns come from counter-based values."""
    rng = np.random.default_rng([seed, 3])
    ed = np.int32 if n_rows < 2**31 else np.int64
    e1 = _nested_ends(rng, n_rows, 1e6, None, ed)
    e2 = _nested_ends(rng, n_rows, 1e4, e1, ed)
    e3 = _nested_ends(rng, n_rows, 1e2, e2, ed)
    c1 = RLE(np.arange(e1.shape[0], dtype=np.int32), e1, n_rows)
    c2 = RLE(_increasing_in_parent(rng, e2, e1, 10_000).astype(np.int32), e2, n_rows)
    c3 = RLE(_increasing_in_parent(rng, e3, e2, 1_000).astype(np.int32), e3, n_rows)
    return c1, c2, c3


def _rle_rows(col: RLE, ranges) -> RLE:
    """The rows of the given sorted disjoint ranges [(start, end), ...] of an
    RLE column, concatenated, as an RLE column (runs cut at range edges)."""
    ends = col.run_ends.astype(np.int64)
    vals, out_ends, base = [], [], 0
    for a, b in ranges:
        i0 = int(np.searchsorted(ends, a, side="right"))
        i1 = int(np.searchsorted(ends, b, side="left"))
        e = np.minimum(ends[i0:i1 + 1], b) - a + base
        vals.append(col.run_values[i0:i1 + 1])
        out_ends.append(e)
        base += b - a
    v = np.concatenate(vals) if vals else col.run_values[:0]
    e = np.concatenate(out_ends) if out_ends else np.zeros(0, np.int64)
    return RLE(v.copy(), e.astype(np.int64), int(base))


def nested_subtable(runs, seed: int, ranges) -> Table:
    """The lean nested table restricted to the given sorted disjoint row
    ranges of the full table (rows concatenated in order): RLE columns cut at
    the range edges, per-row columns evaluated at the original row numbers.
    With ranges [(0, n)] it is the table's first n rows."""
    c1, c2, c3 = (_rle_rows(c, ranges) for c in runs)
    rows = np.concatenate([np.arange(a, b, dtype=np.int64) for a, b in ranges]) if ranges else np.zeros(0, np.int64)
    n = int(rows.shape[0])
    c4 = make_dict(NESTED_DICT4, nested_codes4(seed, runs[2].run_ends, rows), 4)
    c7 = make_packed(nested_row_values(seed, 7, rows), 8, NESTED_BASE7, "i64")
    c8 = make_packed(nested_row_values(seed, 8, rows), 12, NESTED_BASE8, "i64")
    return Table([c1, c2, c3, c4, c7, c8], n, ["c1", "c2", "c3", "c4", "c7", "c8"])


def value_ranges(col: RLE, value: int):
    """Row ranges [(start, end), ...] of the runs of an RLE column holding `value`."""
    ends = col.run_ends.astype(np.int64)
    starts = np.concatenate([[0], ends[:-1]])
    idx = np.flatnonzero(col.run_values == value)
    return [(int(starts[i]), int(ends[i])) for i in idx]


def nested_plan(lo3: int = 200, hi3: int = 699, lean: bool = False) -> Plan:
    m7, m8 = (4, 5) if lean else (6, 7)
    return Plan([Pred(2, "between", lo3, hi3)], [1, 3], [Agg("sum", m7), Agg("sum", m8)])


def tiny_plan(threshold: int = 50) -> Plan:
    return Plan([Pred(0, "lt", threshold)], [1], [Agg("sum", 0), Agg("count")])


def partition_sizes(rng, n_parts: int, lo: float = 1e4, hi: float = 5e7) -> np.ndarray:
    """Partition row counts drawn log-uniform in [lo, hi]."""
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_parts)).astype(np.int64)


def batch_queries(rng, n_queries: int, n_parts: int, lean: bool = True):
    """The batched workload's query list: (partition, kind, plan) with kind
    "tiny" (A < t, t uniform in 0..99, GROUP BY B on the partition's
    two-RLE table) or "nested" (c3 BETWEEN lo AND lo + w on its nested
    table, lean layout unless lean=False), half each, partitions uniform."""
    out = []
    for i in range(n_queries):
        part = int(rng.integers(0, n_parts))
        if i % 2 == 0:
            out.append((part, "tiny", tiny_plan(int(rng.integers(0, 100)))))
        else:
            lo = int(rng.integers(0, 1000))
            hi = min(999, lo + int(rng.integers(0, 1000)))
            out.append((part, "nested", nested_plan(lo, hi, lean)))
    return out


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
