// cq_phases.cuh -- device building blocks shared by the fused query kernels
// (segment mode in cq_query.cu, row mode in cq_row.cu, both in the batch
// kernel of cq_batch.cu): shared-memory layouts, column readers, predicate
// tests, the shared-memory group table and the filter / aggregate phases of
// one tile.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <type_traits>

#include "cq_device.cuh"

namespace cq {

constexpr uint32_t kWin = 128;                           // prefetched run ends / positions per column and tile
constexpr uint32_t kWinBufs = 3;                         // row mode: windows of tiles t, t+1, t+2
constexpr uint32_t kAuxSmemWords = 4096;                 // aux tables up to 16 KB live in shared memory

// ------------------------------------------------------------------ shared-memory layout
struct SmemLayout {
  uint32_t stage, mbar, tkeys, tacc, tacc32, bm, pre, pbm, tcur, win, wcnt, ubm, upre, seg, clist, aux, flags, misc, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Segment mode keeps one bitmap set (built by every warp); row mode double
// buffers bitmaps, start cursors and prefetch windows (built by the helper
// warp one tile ahead).
__host__ __device__ inline SmemLayout smem_layout(const QueryDesc& q) {
  SmemLayout L;
  const uint32_t nwords = q.tile_rows / 32;
  const uint32_t nbuf = q.seg_mode ? 1u : 2u;
  const uint32_t nb = q.n_bitmaps;
  uint32_t off = 0;
  L.stage = off;
  off += q.seg_mode ? 0u : q.stages * q.stage_bytes;
  off = align_up(off, 16);
  L.mbar = off;
  off += 8u * (q.seg_mode ? 0u : q.stages);
  off = align_up(off, 16);
  L.tkeys = off;
  off += q.table_dense ? 0u : (q.ghash ? 8u : 4u) * q.table_slots;
  off = align_up(off, 16);
  L.tacc = off;
  off += 8u * q.n_sw * q.table_slots;
  L.tacc32 = off;
  off += 4u * q.n_sw32 * q.table_slots;
  off = align_up(off, 16);
  L.bm = off;
  off += 4u * nwords * nb * nbuf;
  L.pre = off;
  off += 4u * (nwords + 1) * nb * nbuf;
  L.pbm = off;
  off += 4u * nwords * q.n_pbm * nbuf;
  off = align_up(off, 8);
  L.tcur = off;
  off += 8u * kMaxBitmapCols * nbuf;
  // row mode: per window buffer and bitmap column, kWin run ends / positions
  // followed by the kWin values of the same runs / listed rows
  // segment mode: the next boundary of each bitmap column (long-segment
  // test); walked by runs: each thread's cursor, boundary and value per column
  L.win = off;
  off += q.seg_mode ? (q.run_walk ? 24u * nb * kThreads : 8u * kMaxBitmapCols) : 16u * kWin * nb * kWinBufs;
  L.wcnt = off;
  off += 4u * kMaxBitmapCols * kWinBufs;
  L.ubm = off;
  off += q.seg_mode ? 4u * nwords : 0u;
  L.upre = off;
  off += q.seg_mode ? 4u * (nwords + 1) : 0u;
  L.seg = off;
  off += q.seg_mode ? 2u * (q.tile_rows + 2) : 0u;
  off = align_up(off, 16);
  L.clist = off;
  off += 2u * q.tile_rows;
  off = align_up(off, 16);
  L.aux = off;
  off += q.aux_words <= kAuxSmemWords ? 4u * q.aux_words : 0u;
  off = align_up(off, 16);
  L.flags = off;
  off += 4u * 2 * kMaxBitmapCols;
  L.misc = off;
  off += 4u * 8;
  L.total = align_up(off, 128);
  return L;
}

struct Smem {
  uint8_t* stage;
  uint64_t* mbar;
  uint32_t* tkeys;                 // shared-table keys: 32-bit dense gids ...
  unsigned long long* tkeys64;     // ... or 64-bit packed keys (global hash table), same words
  unsigned long long* tacc;
  unsigned* tacc32;
  uint32_t* bm;
  uint32_t* pre;
  uint32_t* pbm;   // row mode: tile pass bitmaps [buffer][slot][nwords]
  unsigned long long* tcur;
  uint8_t* win;
  uint32_t* wcnt;  // entries held by each window [buffer][column] (segment mode: zeros)
  uint32_t* ubm;
  uint32_t* upre;
  uint16_t* seg;
  uint16_t* clist;
  uint32_t* aux;
  int* flags;   // segment mode: [j] column done, [kMaxBitmapCols + j] run ends exactly at the tile end
  int* misc;    // 0 occupancy, 2 segments of the tile
};

extern __shared__ __align__(128) uint8_t g_smem[];

__device__ __forceinline__ Smem carve(const QueryDesc& q) {
  const SmemLayout L = smem_layout(q);
  Smem s;
  s.stage = g_smem + L.stage;
  s.mbar = reinterpret_cast<uint64_t*>(g_smem + L.mbar);
  s.tkeys = reinterpret_cast<uint32_t*>(g_smem + L.tkeys);
  s.tkeys64 = reinterpret_cast<unsigned long long*>(g_smem + L.tkeys);
  s.tacc = reinterpret_cast<unsigned long long*>(g_smem + L.tacc);
  s.tacc32 = reinterpret_cast<unsigned*>(g_smem + L.tacc32);
  s.bm = reinterpret_cast<uint32_t*>(g_smem + L.bm);
  s.pre = reinterpret_cast<uint32_t*>(g_smem + L.pre);
  s.pbm = reinterpret_cast<uint32_t*>(g_smem + L.pbm);
  s.tcur = reinterpret_cast<unsigned long long*>(g_smem + L.tcur);
  s.win = g_smem + L.win;
  s.wcnt = reinterpret_cast<uint32_t*>(g_smem + L.wcnt);
  s.ubm = reinterpret_cast<uint32_t*>(g_smem + L.ubm);
  s.upre = reinterpret_cast<uint32_t*>(g_smem + L.upre);
  s.seg = reinterpret_cast<uint16_t*>(g_smem + L.seg);
  s.clist = reinterpret_cast<uint16_t*>(g_smem + L.clist);
  s.aux = reinterpret_cast<uint32_t*>(g_smem + L.aux);
  s.flags = reinterpret_cast<int*>(g_smem + L.flags);
  s.misc = reinterpret_cast<int*>(g_smem + L.misc);
  return s;
}

// Everything a column reader needs about the tile being processed.
struct TileView {
  const uint32_t* bm;                // bitmaps of this tile [n_bitmaps][nwords]
  const uint32_t* pre;               // word prefix popcounts [n_bitmaps][nwords + 1]
  const unsigned long long* cur;     // first run / position of each bitmap column in this tile
  const uint8_t* win;                // window set of this tile (row mode), see win_value
  const uint32_t* pbm;               // pass bitmaps of this tile (row mode) [slot][nwords]
  const uint32_t* wn;                // entries in each column's window (0: none)
  const uint8_t* stage;              // staged row-level columns of this tile
  const uint32_t* aux;               // predicate / key tables (shared or global memory)
  uint32_t nwords;
  unsigned long long line_base;      // line mode: first run whose line is not flushed yet
};

// ------------------------------------------------------------------ dispatch
template <int V>
using IC = std::integral_constant<int, V>;

template <class F>
__device__ __forceinline__ void dispatch_enc(uint8_t enc, F&& f) {
  switch (enc) {
    case ENC_PLAIN: f(IC<ENC_PLAIN>()); break;
    case ENC_PACKED: f(IC<ENC_PACKED>()); break;
    case ENC_DICT: f(IC<ENC_DICT>()); break;
    case ENC_RLE: f(IC<ENC_RLE>()); break;
    default: f(IC<ENC_INDEX>()); break;
  }
}

// Encodings that can occur: segment mode has only RLE and index columns.
template <bool SEG, class F>
__device__ __forceinline__ void dispatch_col(uint8_t enc, F&& f) {
  if constexpr (SEG) {
    if (enc == ENC_RLE) f(IC<ENC_RLE>());
    else f(IC<ENC_INDEX>());
  } else {
    dispatch_enc(enc, f);
  }
}

// Predicate kinds evaluated per row; a narrow (32-bit) variant of each
// comparison kind is used when the planner proved the column's raw values fit.
enum { PT_RANGE = 0, PT_NE = 1, PT_BITMAP = 2, PT_LIST = 3, PT_RANGE32 = 4, PT_NE32 = 5, PT_BITMAP32 = 6 };

template <class F>
__device__ __forceinline__ void dispatch_test(const PredDesc& p, F&& f) {
  if (p.n32) {
    switch (p.kind) {
      case PK_RANGE: f(IC<PT_RANGE32>()); return;
      case PK_NE: f(IC<PT_NE32>()); return;
      case PK_BITMAP: f(IC<PT_BITMAP32>()); return;
      default: break;
    }
  }
  switch (p.kind) {
    case PK_RANGE: f(IC<PT_RANGE>()); break;
    case PK_NE: f(IC<PT_NE>()); break;
    case PK_BITMAP: f(IC<PT_BITMAP>()); break;
    default: f(IC<PT_LIST>()); break;
  }
}

// ------------------------------------------------------------------ column readers
// Value of the tile's k-th run (RLE) or listed row (index) of column c: from
// the shared-memory window the helper warp prefetched for this tile when it
// holds entry k, else from global memory.
__device__ __forceinline__ long long win_value(const ColDesc& c, const TileView& t, uint32_t k) {
  if (k < t.wn[c.bslot]) {
    const uint8_t* v = t.win + (size_t)c.bslot * kWin * 16 + kWin * 8;
    return c.v64 ? reinterpret_cast<const long long*>(v)[k] : (long long)reinterpret_cast<const int*>(v)[k];
  }
  return ldg_val(c.vals, t.cur[c.bslot] + k, c.v64);
}

// Raw value of column c at tile row o (the logical value for RLE / index /
// plain columns; the unsigned field for dictionary codes and, when
// raw_is_offset, bit-packed offsets).
template <int ENC>
__device__ __forceinline__ long long col_raw(const ColDesc& c, const TileView& t, uint32_t o) {
  if constexpr (ENC == ENC_PLAIN) {
    const uint8_t* p = t.stage + c.stage_off;
    return c.v64 ? reinterpret_cast<const long long*>(p)[o] : (long long)reinterpret_cast<const int*>(p)[o];
  } else if constexpr (ENC == ENC_PACKED || ENC == ENC_DICT) {
    const uint64_t f = extract_field(reinterpret_cast<const uint32_t*>(t.stage + c.stage_off), o, c.bw);
    return c.raw_is_offset ? (long long)f : (long long)(f + (uint64_t)c.base);
  } else if constexpr (ENC == ENC_RLE) {
    const uint32_t* B = t.bm + c.bslot * t.nwords;
    const uint32_t* P = t.pre + c.bslot * (t.nwords + 1);
    return win_value(c, t, rank_incl(B, P, o));
  } else {  // ENC_INDEX
    const uint32_t* B = t.bm + c.bslot * t.nwords;
    const uint32_t wv = B[o >> 5];
    if (!((wv >> (o & 31)) & 1u)) return c.base;
    const uint32_t* P = t.pre + c.bslot * (t.nwords + 1);
    return win_value(c, t, P[o >> 5] + __popc(wv & ((1u << (o & 31)) - 1u)));
  }
}

// 32-bit raw value; valid only for columns the planner marked narrow.
template <int ENC>
__device__ __forceinline__ int col_raw32(const ColDesc& c, const TileView& t, uint32_t o) {
  if constexpr (ENC == ENC_PLAIN) {
    return reinterpret_cast<const int*>(t.stage + c.stage_off)[o];
  } else if constexpr (ENC == ENC_PACKED || ENC == ENC_DICT) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(t.stage + c.stage_off);
    const uint32_t bit = o * (uint32_t)c.bw;
    const uint32_t q = bit >> 5;
    const uint32_t v = __funnelshift_r(w[q], w[q + 1], bit & 31);
    return (int)(c.bw >= 32 ? v : (v & ((1u << c.bw) - 1u)));
  } else if constexpr (ENC == ENC_RLE) {
    const uint32_t* B = t.bm + c.bslot * t.nwords;
    const uint32_t* P = t.pre + c.bslot * (t.nwords + 1);
    return (int)win_value(c, t, rank_incl(B, P, o));
  } else {
    const uint32_t* B = t.bm + c.bslot * t.nwords;
    const uint32_t wv = B[o >> 5];
    if (!((wv >> (o & 31)) & 1u)) return (int)c.base;
    const uint32_t* P = t.pre + c.bslot * (t.nwords + 1);
    return (int)win_value(c, t, P[o >> 5] + __popc(wv & ((1u << (o & 31)) - 1u)));
  }
}

__device__ __forceinline__ long long col_value(const ColDesc& c, const TileView& t, uint32_t o) {
  switch (c.enc) {
    case ENC_PLAIN: return col_raw<ENC_PLAIN>(c, t, o);
    case ENC_PACKED: return col_raw<ENC_PACKED>(c, t, o);
    case ENC_DICT: return col_raw<ENC_DICT>(c, t, o);
    case ENC_RLE: return col_raw<ENC_RLE>(c, t, o);
    default: return col_raw<ENC_INDEX>(c, t, o);
  }
}

// Index column at o: listed? and value.
__device__ __forceinline__ bool index_lookup(const ColDesc& c, const TileView& t, uint32_t o, long long* v) {
  const uint32_t* B = t.bm + c.bslot * t.nwords;
  const uint32_t wv = B[o >> 5];
  if (!((wv >> (o & 31)) & 1u)) return false;
  const uint32_t* P = t.pre + c.bslot * (t.nwords + 1);
  *v = win_value(c, t, P[o >> 5] + __popc(wv & ((1u << (o & 31)) - 1u)));
  return true;
}

// ------------------------------------------------------------------ predicates and keys
template <int K>
__device__ __forceinline__ bool pred_test(const PredDesc& p, const uint32_t* aux, long long v) {
  if constexpr (K == PT_RANGE) {
    return v >= p.lo && v <= p.hi;
  } else if constexpr (K == PT_NE) {
    return v != p.lo;
  } else if constexpr (K == PT_BITMAP) {
    if (v < p.lo || v > p.hi) return false;
    const unsigned long long d = (unsigned long long)(v - p.lo);
    return (aux[p.aux_off + (uint32_t)(d >> 5)] >> (d & 31)) & 1u;
  } else {  // PT_LIST
    const long long* L = reinterpret_cast<const long long*>(aux + p.aux_off);
    uint32_t lo = 0, hi = p.aux_len;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (L[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    return lo < p.aux_len && L[lo] == v;
  }
}

template <int K>
__device__ __forceinline__ bool pred_test32(const PredDesc& p, const uint32_t* aux, int v) {
  if constexpr (K == PT_RANGE32) {
    return (unsigned)v - (unsigned)p.lo32 <= (unsigned)p.hi32 - (unsigned)p.lo32;
  } else if constexpr (K == PT_NE32) {
    return v != p.lo32;
  } else {  // PT_BITMAP32
    const unsigned d = (unsigned)v - (unsigned)p.lo32;
    if (d > (unsigned)p.hi32 - (unsigned)p.lo32) return false;
    return (aux[p.aux_off + (d >> 5)] >> (d & 31)) & 1u;
  }
}

// digit of key k for raw value v; false when v is outside the key's domain
__device__ __forceinline__ bool key_digit(const KeyDesc& k, const uint32_t* aux, long long v,
                                          unsigned long long* digit) {
  const unsigned long long d = (unsigned long long)v - (unsigned long long)k.kmin;
  if (!k.remap) {
    if (v < k.kmin || d >= k.card) return false;
    *digit = d;
    return true;
  }
  if (v < k.kmin || d >= 32ull * k.aux_len) return false;
  const uint32_t w = aux[k.aux_off + (uint32_t)(d >> 5)];
  if (!((w >> (d & 31)) & 1u)) return false;
  *digit = aux[k.prefix_off + (uint32_t)(d >> 5)] + __popc(w & ((1u << (d & 31)) - 1u));
  return true;
}

// A predicate on one raw value (the helper's once-per-run evaluation),
// complemented when the predicate is negated.
__device__ __forceinline__ bool pred_eval(const PredDesc& p, const uint32_t* aux, long long v) {
  bool r;
  switch (p.kind) {
    case PK_RANGE: r = pred_test<PT_RANGE>(p, aux, v); break;
    case PK_NE: r = pred_test<PT_NE>(p, aux, v); break;
    case PK_BITMAP: r = pred_test<PT_BITMAP>(p, aux, v); break;
    case PK_LIST: r = pred_test<PT_LIST>(p, aux, v); break;
    case PK_FALSE: r = false; break;
    default: r = true; break;
  }
  return r != (p.neg != 0);
}

// key_digit for a key whose raw values are read in 32 bits and whose kmin
// lies within +-2^30 (so v - kmin cannot wrap into the digit range).
__device__ __forceinline__ bool key_digit32(const KeyDesc& k, const uint32_t* aux, int v, unsigned long long* digit) {
  const uint32_t d = (uint32_t)v - (uint32_t)(int)k.kmin;
  if (!k.remap) {
    if (d >= k.card) return false;
    *digit = d;
    return true;
  }
  if (d >= 32u * k.aux_len) return false;
  const uint32_t w = aux[k.aux_off + (d >> 5)];
  if (!((w >> (d & 31)) & 1u)) return false;
  *digit = aux[k.prefix_off + (d >> 5)] + __popc(w & ((1u << (d & 31)) - 1u));
  return true;
}

// The column whose bitmap slot is j.
__device__ __forceinline__ const ColDesc& bitmap_col(const QueryDesc& q, int j) {
  int idx = 0;
  for (int c = 0; c < q.n_cols; ++c)
    if (q.cols[c].bslot == j) idx = c;
  return q.cols[idx];
}

// First device error wins; its detail (what, where, value) is kept for the host.
__device__ __forceinline__ void report(const QueryDesc& q, int code, unsigned long long what,
                                       unsigned long long where, unsigned long long value) {
  if (atomicCAS(q.err, 0, code) == 0) {
    q.err_info[0] = what;
    q.err_info[1] = where;
    q.err_info[2] = value;
  }
}

// ------------------------------------------------------------------ group table
// Shared-memory group table, structure of arrays over `table_slots` slots: a
// 64-bit word array (SUMs, wide MIN / MAX) and a 32-bit word array (COUNT in
// word 0, MIN / MAX whose values fit 32 bits, listed counts of index columns).

// multiplicative hashing: the top bits of gid * golden ratio select the slot
__device__ __forceinline__ uint32_t hash_gid(uint32_t g, uint32_t log2_slots) {
  return (g * 0x9E3779B1u) >> (32 - log2_slots);
}

// Shared-memory slot of gid, or -1 when the probe limit is hit (caller then
// updates the global accumulators directly).  Dense domains key the table by
// the 32-bit gid, hash domains by the 64-bit packed key.
template <bool GH>
__device__ __forceinline__ int table_slot_t(const QueryDesc& q, const Smem& sm, unsigned long long gid) {
  if (q.table_dense) return (int)gid;
  const uint32_t mask = q.table_slots - 1;
  const uint32_t lg = 31 - __clz(q.table_slots);
  if constexpr (GH) {
    uint32_t h = (uint32_t)((gid * 0x9E3779B97F4A7C15ull) >> (64 - lg)) & mask;
    for (int probe = 0; probe < 32; ++probe) {
      unsigned long long k = sm.tkeys64[h];
      if (k == gid) return (int)h;
      if (k == kEmptyGroup) {
        k = atomicCAS(&sm.tkeys64[h], kEmptyGroup, gid);
        if (k == kEmptyGroup) {
          atomicAdd(&sm.misc[0], 1);
          return (int)h;
        }
        if (k == gid) return (int)h;
      }
      h = (h + 1) & mask;
    }
    return -1;
  }
  const uint32_t g = (uint32_t)gid;
  uint32_t h = hash_gid(g, lg) & mask;
  for (int probe = 0; probe < 32; ++probe) {
    uint32_t k = sm.tkeys[h];
    if (k == g) return (int)h;
    if (k == kEmptyKey) {
      k = atomicCAS(&sm.tkeys[h], kEmptyKey, g);
      if (k == kEmptyKey) {
        atomicAdd(&sm.misc[0], 1);
        return (int)h;
      }
      if (k == g) return (int)h;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

// Index of group gid in the global accumulators: the gid itself in a dense
// domain; in a hash domain the slot of its packed key in the open-addressing
// key table (linear probing from a multiplicative hash, inserting the key;
// keys are never removed).  After kGlobalProbes occupied slots the query
// fails with CQ_ERR_TABLE_FULL (the host then retries with a larger table)
// and -1 is returned: the caller skips the update.
template <bool GH>
__device__ __forceinline__ long long gindex_t(const QueryDesc& q, unsigned long long gid) {
  if constexpr (!GH) return (long long)gid;
  const unsigned long long mask = q.n_groups - 1;
  const uint32_t lg = 63 - __clzll((long long)q.n_groups);
  unsigned long long h = lg ? ((gid * 0x9E3779B97F4A7C15ull) >> (64 - lg)) & mask : 0ull;
  for (int probe = 0; probe < kGlobalProbes; ++probe) {
    unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&q.gkeys[h]);
    if (k == gid) return (long long)h;
    if (k == kEmptyGroup) {
      k = atomicCAS(&q.gkeys[h], kEmptyGroup, gid);
      if (k == kEmptyGroup || k == gid) return (long long)h;
    }
    h = (h + 1) & mask;
  }
  if (atomicCAS(q.err, 0, (int)CQ_ERR_TABLE_FULL) == 0) {
    q.err_info[0] = 4;
    q.err_info[1] = q.n_groups;
    q.err_info[2] = gid;
  }
  return -1;
}

// (the descriptor's domain kind read at run time)
__device__ __forceinline__ int table_slot(const QueryDesc& q, const Smem& sm, unsigned long long gid) {
  return q.ghash ? table_slot_t<true>(q, sm, gid) : table_slot_t<false>(q, sm, gid);
}
__device__ __forceinline__ long long gindex(const QueryDesc& q, unsigned long long gid) {
  return q.ghash ? gindex_t<true>(q, gid) : (long long)gid;
}

__device__ __forceinline__ unsigned long long* gword(const QueryDesc& q, uint32_t w, uint32_t gid) {
  return q.gacc + (size_t)w * q.n_groups + gid;
}

__device__ __forceinline__ unsigned long long* sword(const QueryDesc& q, const Smem& sm, uint32_t w, int slot) {
  return &sm.tacc[(size_t)w * q.table_slots + slot];
}

__device__ __forceinline__ int* sword32(const QueryDesc& q, const Smem& sm, uint32_t w, int slot) {
  return reinterpret_cast<int*>(&sm.tacc32[(size_t)w * q.table_slots + slot]);
}

__device__ __forceinline__ unsigned* scount(const QueryDesc& q, const Smem& sm, int slot) {
  return &sm.tacc32[slot];
}

// 32-bit word of an index column's listed count
__device__ __forceinline__ unsigned* slisted(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot) {
  return reinterpret_cast<unsigned*>(sword32(q, sm, a.sw32 + (a.w32 ? 1 : 0), slot));
}

// 128-bit value of (v - base) for an index column's listed row
__device__ __forceinline__ I128 index_delta(long long v, long long base) {
  I128 x;
  x.lo = (unsigned long long)v - (unsigned long long)base;
  x.hi = (v < 0 ? -1ll : 0ll) - (base < 0 ? -1ll : 0ll) - ((unsigned long long)v < (unsigned long long)base ? 1ll : 0ll);
  return x;
}

// Narrow SUM accumulator: one 64-bit shared word used as a low unsigned and a
// high signed 32-bit half.  The old low half returned by the 32-bit atomic
// tells whether this addend carried, so the word always holds the exact
// two's-complement sum while only native 32-bit shared atomics are used.
__device__ __forceinline__ void smem_add64(unsigned long long* w, long long x) {
  unsigned* p = reinterpret_cast<unsigned*>(w);
  const unsigned xl = (unsigned)(unsigned long long)x;
  const unsigned old = atomicAdd(p, xl);
  const unsigned h = (unsigned)((unsigned long long)x >> 32) + ((old + xl) < old ? 1u : 0u);
  if (h) atomicAdd(p + 1, h);
}

// Split SUM accumulator (s32 == 3): x < 2^31 goes to two 32-bit limb words,
// its low kSplitBits bits and the rest, with atomics whose result is unused.
// lo and hi are the accumulator's two words (word sw32 and sw32 + 1 of the slot).
__device__ __forceinline__ void split_add(int* lo, int* hi, unsigned x) {
  atomicAdd(reinterpret_cast<unsigned*>(lo), x & ((1u << kSplitBits) - 1u));
  if (x >> kSplitBits) atomicAdd(reinterpret_cast<unsigned*>(hi), x >> kSplitBits);
}

// Value of a split SUM accumulator.
__device__ __forceinline__ long long split_value(const int* lo, const int* hi) {
  return (long long)(unsigned)*lo + ((long long)(unsigned)*hi << kSplitBits);
}

// Add a 128-bit contribution to a SUM accumulator in shared memory (slot >= 0)
// or straight into the global limbs of global index gi (see gindex).
__device__ __forceinline__ void sum_add(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot, uint32_t gi,
                                        I128 x) {
  if (slot >= 0) {
    if (a.s32 == 3) split_add(sword32(q, sm, a.sw32, slot), sword32(q, sm, a.sw32 + 1, slot), (unsigned)x.lo);
    else if (a.s32) atomicAdd(reinterpret_cast<unsigned*>(sword32(q, sm, a.sw32, slot)), (unsigned)x.lo);
    else if (!a.wide) smem_add64(sword(q, sm, a.sw, slot), (long long)x.lo);
    else atomic_add_i128(sword(q, sm, a.sw, slot), sword(q, sm, a.sw + 1, slot), x);
  } else {
    global_add_limbs(gword(q, a.gw, gi), gword(q, a.gw + 1, gi), gword(q, a.gw + 2, gi), x);
  }
}

__device__ __forceinline__ void minmax_add(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot,
                                           uint32_t gi, long long v, bool is_min) {
  if (slot >= 0) {
    // read first: most values do not improve the extreme, and a plain read
    // is cheaper than an atomic (a stale read only costs an extra atomic)
    if (a.w32) {
      int* p = sword32(q, sm, a.sw32, slot);
      const int cur = *reinterpret_cast<volatile int*>(p);
      if (is_min ? (int)v < cur : (int)v > cur) {
        if (is_min) atomicMin(p, (int)v);
        else atomicMax(p, (int)v);
      }
    } else {
      long long* p = reinterpret_cast<long long*>(sword(q, sm, a.sw, slot));
      const long long cur = *reinterpret_cast<volatile long long*>(p);
      if (is_min ? v < cur : v > cur) {
        if (is_min) atomicMin(p, v);
        else atomicMax(p, v);
      }
    }
  } else {
    if (is_min) atomicMin(reinterpret_cast<long long*>(gword(q, a.gw, gi)), v);
    else atomicMax(reinterpret_cast<long long*>(gword(q, a.gw, gi)), v);
  }
}

__device__ __forceinline__ void reset_slot(const QueryDesc& q, const Smem& sm, uint32_t s) {
  *scount(q, sm, s) = 0;
  for (int i = 0; i < q.n_aggs; ++i) {
    const AggDesc& a = q.aggs[i];
    switch (a.kind) {
      case AK_SUM:
      case AK_ISUM:
      case AK_SUM2:
      case AK_ISUM2:
        if (a.s32) {
          *sword32(q, sm, a.sw32, s) = 0;
          if (a.s32 == 3) *sword32(q, sm, a.sw32 + 1, s) = 0;
        } else {
          *sword(q, sm, a.sw, s) = 0;
          if (a.wide) *sword(q, sm, a.sw + 1, s) = 0;
        }
        break;
      case AK_MIN:
      case AK_IMIN:
      case AK_MAX:
      case AK_IMAX: {
        const bool mn = a.kind == AK_MIN || a.kind == AK_IMIN;
        if (a.w32) *sword32(q, sm, a.sw32, s) = mn ? INT_MAX : INT_MIN;
        else *sword(q, sm, a.sw, s) = mn ? (unsigned long long)LLONG_MAX : (unsigned long long)LLONG_MIN;
        if (a.kind == AK_IMIN || a.kind == AK_IMAX) *slisted(q, sm, a, s) = 0;
        break;
      }
      default:
        break;
    }
  }
  if (!q.table_dense && !q.line_mode) {   // (line mode keeps line digits there)
    if (q.ghash) sm.tkeys64[s] = kEmptyGroup;
    else sm.tkeys[s] = kEmptyKey;
  }
}

// Add shared slot s (cnt rows counted) into the global accumulators of group
// index gid and clear the slot.
__device__ inline void flush_slot(const QueryDesc& q, const Smem& sm, uint32_t s, unsigned cnt, uint32_t gid) {
  atomicAdd(gword(q, 0, gid), (unsigned long long)cnt);
  for (int i = 0; i < q.n_aggs; ++i) {
    const AggDesc& a = q.aggs[i];
    switch (a.kind) {
      case AK_SUM:
      case AK_ISUM:
      case AK_SUM2:
      case AK_ISUM2: {
        I128 x;
        if (a.s32 == 3) {
          x = sext(split_value(sword32(q, sm, a.sw32, s), sword32(q, sm, a.sw32 + 1, s)));
        } else if (a.s32 == 1) {
          x = sext((long long)(unsigned)*sword32(q, sm, a.sw32, s));
        } else if (a.s32 == 2) {
          x = sext((long long)*sword32(q, sm, a.sw32, s));
        } else if (a.wide) {
          x.lo = *sword(q, sm, a.sw, s);
          x.hi = (long long)*sword(q, sm, a.sw + 1, s);
        } else {
          x = sext((long long)*sword(q, sm, a.sw, s));
        }
        global_add_limbs(gword(q, a.gw, gid), gword(q, a.gw + 1, gid), gword(q, a.gw + 2, gid), x);
        break;
      }
      case AK_MIN:
      case AK_IMIN: {
        const long long v = a.w32 ? (long long)*sword32(q, sm, a.sw32, s) : (long long)*sword(q, sm, a.sw, s);
        if (v != (a.w32 ? (long long)INT_MAX : LLONG_MAX)) atomicMin(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
        break;
      }
      case AK_MAX:
      case AK_IMAX: {
        const long long v = a.w32 ? (long long)*sword32(q, sm, a.sw32, s) : (long long)*sword(q, sm, a.sw, s);
        if (v != (a.w32 ? (long long)INT_MIN : LLONG_MIN)) atomicMax(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
        break;
      }
      default:
        break;
    }
    if (a.kind == AK_IMIN || a.kind == AK_IMAX) {
      const unsigned lc = *slisted(q, sm, a, s);
      if (lc) atomicAdd(gword(q, a.gw + 1, gid), (unsigned long long)lc);
    }
  }
  reset_slot(q, sm, s);
}

// Group id of run-line slot s (line mode): key 0's digit of the line's run
// (recorded in the line's digit word when the run's tile was aggregated, see
// line_digits), times its stride, plus the slot's inner digits (the slot's
// place in the line, un-swizzled).
__device__ __forceinline__ bool line_group(const QueryDesc& q, const Smem& sm, uint32_t s, unsigned long long* gid) {
  const uint32_t line = s / q.line_inner, inner = (s - line * q.line_inner) ^ (line & q.line_swz);
  if (line >= (1u << q.line_log2)) return false;
  const unsigned long long d = sm.tkeys64[line];
  if (d == ~0ull) return false;
  *gid = d * q.keys[0].stride + inner;
  return true;
}

// Flush the shared table into the global accumulators and clear it.
__device__ inline void flush_table(const QueryDesc& q, const Smem& sm) {
  const uint32_t S = q.table_slots;
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
    const unsigned cnt = *scount(q, sm, s);
    if (cnt == 0) {
      if (!q.table_dense && !q.line_mode) {
        if (q.ghash) sm.tkeys64[s] = kEmptyGroup;
        else sm.tkeys[s] = kEmptyKey;
      }
      continue;
    }
    // a counted slot always holds its key; one that does not (or a key
    // outside the domain) is reported and dropped, never used as an index
    unsigned long long key = 0;
    bool bad;
    if (q.line_mode) {
      bad = !line_group(q, sm, s, &key);
      bad = bad || key >= q.n_groups;
    } else {
      key = q.table_dense ? s : (q.ghash ? sm.tkeys64[s] : (unsigned long long)sm.tkeys[s]);
      bad = q.ghash ? key == kEmptyGroup : key >= q.n_groups;
    }
    if (bad) {
      report(q, CQ_ERR_INVALID_ARG, 4ull, s, key);
      reset_slot(q, sm, s);
      continue;
    }
    const long long g = q.ghash ? gindex(q, key) : (long long)key;
    if (g < 0) {   // global hash table full: the query fails, the host retries larger
      reset_slot(q, sm, s);
      continue;
    }
    flush_slot(q, sm, s, cnt, (uint32_t)g);
  }
}

// Line mode: record key 0's digit for the lines of a tile's runs, ordinals
// cur .. cur + nset (warp 0 of the compute warps; ~0 when a value lies outside
// the key's domain, which the flush then reports).
__device__ inline void line_digits(const QueryDesc& q, const Smem& sm, const TileView& t, unsigned long long cur,
                                   uint32_t nset) {
  const uint32_t lines = 1u << q.line_log2;
  const KeyDesc& k = q.keys[0];
  for (uint32_t r = threadIdx.x & 31; r <= nset; r += 32) {
    unsigned long long d;
    if (!key_digit(k, t.aux, win_value(q.cols[k.col], t, r), &d)) d = ~0ull;
    sm.tkeys64[(uint32_t)(cur + r) & (lines - 1u)] = d;
  }
}

// ------------------------------------------------------------------ tile phases
// Bit g: item (wbase + g * gstride + lane) passes test p (before any
// complement).  Segment mode reads only the items still set in `live`.
template <bool SEG, int GPW>
__device__ __forceinline__ uint32_t filter_tests(const QueryDesc& q, const TileView& t, const uint16_t* seg,
                                                 const PredDesc& p, uint32_t wbase, uint32_t gstride, uint32_t live) {
  const int lane = threadIdx.x & 31;
  const ColDesc& c = q.cols[p.col];
  uint32_t m = 0;
  dispatch_col<SEG>(c.enc, [&](auto et) {
    dispatch_test(p, [&](auto kt) {
      constexpr int E = decltype(et)::value;
      constexpr int K = decltype(kt)::value;
      if constexpr (SEG) {
#pragma unroll 2
        for (int g = 0; g < GPW; ++g) {
          if (!((live >> g) & 1u)) continue;
          const uint32_t o = (uint32_t)seg[wbase + g * gstride + lane];
          bool ok;
          if constexpr (K >= PT_RANGE32) ok = pred_test32<K>(p, t.aux, col_raw32<E>(c, t, o));
          else ok = pred_test<K>(p, t.aux, col_raw<E>(c, t, o));
          m |= (ok ? 1u : 0u) << g;
        }
      } else {
        // rows of a tile are always readable (stale beyond the last row,
        // masked by `valid`), so every group is evaluated without branches
        // and the unrolled loads of several groups overlap
#pragma unroll 4
        for (int g = 0; g < GPW; ++g) {
          const uint32_t o = wbase + g * gstride + lane;
          bool ok;
          if constexpr (K >= PT_RANGE32) ok = pred_test32<K>(p, t.aux, col_raw32<E>(c, t, o));
          else ok = pred_test<K>(p, t.aux, col_raw<E>(c, t, o));
          m |= (ok ? 1u : 0u) << g;
        }
      }
    });
  });
  return m;
}

// Filter: bit g of the result says item (wbase + g * gstride + lane) passes
// the filter, a conjunction of clauses (Section 5: AND, OR, NOT).  Callers
// deal 32-item groups to warps round-robin (wbase = 32 * warp, gstride = 32 *
// warps), so that the clustered passing rows of sorted data spread evenly
// over the warps.  Items are rows (row mode) or aligned segments (segment
// mode, item -> first row through seg[]).  Predicates are evaluated one at a
// time over all of the warp's items, with the column / test dispatch hoisted
// out of the item loop: bit g of `m` is the item's result (complemented for a
// negated predicate; a pass bitmap already holds the complement), AND-ed into
// the mask for a predicate alone in its clause, else OR-ed into `acc`, which
// the clause's last member ANDs in.
template <bool SEG, int GPW>
__device__ __forceinline__ uint32_t phase_filter(const QueryDesc& q, const TileView& t, const uint16_t* seg,
                                                 uint32_t wbase, uint32_t gstride, uint32_t n_items) {
  const int lane = threadIdx.x & 31;
  uint32_t valid = 0;
#pragma unroll
  for (int g = 0; g < GPW; ++g) valid |= (wbase + g * gstride + lane < n_items ? 1u : 0u) << g;
  uint32_t pm = valid, acc = 0;
  for (int oi = 0; oi < q.n_preds; ++oi) {
    if (!__any_sync(0xFFFFFFFFu, pm != 0)) break;
    const PredDesc& p = q.preds[oi];
    uint32_t m = 0;
    if (!SEG && p.pbm != 0xFF) {
      // evaluated once per run by the helper warp: one bit per row
      const uint32_t* PB = t.pbm + (size_t)p.pbm * t.nwords;
#pragma unroll 4
      for (int g = 0; g < GPW; ++g) m |= ((PB[(wbase + g * gstride) >> 5] >> lane) & 1u) << g;
    } else if (p.kind == PK_TRUE || p.kind == PK_FALSE) {
      m = p.kind == PK_TRUE ? ~0u : 0u;
    } else {
      m = filter_tests<SEG, GPW>(q, t, seg, p, wbase, gstride, pm);
      if (p.neg) m = ~m;
    }
    if (p.clause == PC_ALONE) {
      pm &= m;
    } else {
      acc |= m;
      if (p.clause == PC_LAST) {
        pm &= acc;
        acc = 0;
      }
    }
  }
  return pm & valid;
}

// Compact the passing items of this warp into list[] (item indices).
template <int GPW>
__device__ __forceinline__ uint32_t compact(uint32_t pm, uint32_t wbase, uint32_t gstride, uint16_t* list) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t n = 0;
#pragma unroll
  for (int g = 0; g < GPW; ++g) {
    const bool ok = (pm >> g) & 1u;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) list[n + __popc(bal & lt)] = (uint16_t)(wbase + g * gstride + lane);
    n += __popc(bal);
  }
  __syncwarp();
  return n;
}

// One aggregate's update for one item (slot >= 0: shared table; else global).
// Row mode items are single rows (len 1); segment items weigh by length.
// col (expr) col2 of two actual values; the planner keeps the result within
// int64 (unsigned arithmetic: no undefined overflow).
__device__ __forceinline__ long long expr_apply(uint8_t e, long long x, long long y) {
  const unsigned long long a = (unsigned long long)x, b = (unsigned long long)y;
  return (long long)(e == EXPR_ADD ? a + b : (e == EXPR_SUB ? a - b : a * b));
}

template <bool SEG>
__device__ __forceinline__ void agg_item(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot,
                                         uint32_t gi, long long v, uint32_t len) {
  if (a.kind == AK_SUM) sum_add(q, sm, a, slot, gi, SEG ? mul_s64(v, (long long)len) : sext(v));
  else if (a.kind == AK_SUM2) sum_add(q, sm, a, slot, gi, SEG ? mul_s64(v * v, (long long)len) : sext(v * v));
  else minmax_add(q, sm, a, slot, gi, v, a.kind == AK_MIN);
}

// Aggregate: passing items in batches of 32 * MI per warp, MI per lane.  Keys,
// slots and every aggregate are separate passes over the batch with the key /
// aggregate dispatch hoisted out, so the MI items of a lane form independent
// chains.  Each item updates its group's shared slot with native 32-bit
// shared atomics (or the global accumulators when the table has no free slot
// within the probe limit).  A single-group query reduces across the warp
// first and one lane updates.
template <bool SEG, int MI>
__device__ __forceinline__ void phase_aggregate(const QueryDesc& q, const Smem& sm, const TileView& t,
                                                const uint16_t* seg, const uint16_t* list, uint32_t n_pass,
                                                unsigned long long tile_row0) {
  const int lane = threadIdx.x & 31;
  const bool one_group = q.n_groups == 1;
  for (uint32_t j0 = 0; j0 < n_pass; j0 += 32 * MI) {
    uint32_t o[MI], len[MI], gi[MI];
    unsigned long long gid[MI];
    int slot[MI];
    bool act[MI];
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const uint32_t j = j0 + m * 32 + lane;
      act[m] = j < n_pass;
      const uint32_t itm = act[m] ? list[j] : list[j0];
      if (SEG) {
        o[m] = seg[itm];
        len[m] = act[m] ? (uint32_t)seg[itm + 1] - o[m] : 0u;
      } else {
        o[m] = itm;
        len[m] = act[m] ? 1u : 0u;
      }
      gid[m] = 0;
      gi[m] = 0;
      slot[m] = -1;
    }
    // ---- group ids
    for (int ki = 0; ki < q.n_keys; ++ki) {
      const KeyDesc& k = q.keys[ki];
      const ColDesc& c = q.cols[k.col];
      dispatch_col<SEG>(c.enc, [&](auto et) {
        constexpr int E = decltype(et)::value;
        if (k.n32) {
#pragma unroll
          for (int m = 0; m < MI; ++m) {
            const int v = col_raw32<E>(c, t, o[m]);
            unsigned long long d;
            if (key_digit32(k, t.aux, v, &d)) {
              gid[m] += d * k.stride;
            } else if (act[m]) {
              act[m] = false;
              report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)ki << 8), tile_row0 + o[m],
                     (unsigned long long)(long long)v);
            }
          }
          return;
        }
#pragma unroll
        for (int m = 0; m < MI; ++m) {
          const long long v = col_raw<E>(c, t, o[m]);
          unsigned long long d;
          if (key_digit(k, t.aux, v, &d)) {
            gid[m] += d * k.stride;
          } else if (act[m]) {
            act[m] = false;
            report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)ki << 8), tile_row0 + o[m], (unsigned long long)v);
          }
        }
      });
    }
    // ---- slots and COUNT
    if (one_group) {
      uint32_t tot = 0;
#pragma unroll
      for (int m = 0; m < MI; ++m) tot += act[m] ? len[m] : 0u;
      tot = __reduce_add_sync(0xFFFFFFFFu, tot);
      if (lane == 0) atomicAdd(scount(q, sm, 0), tot);
#pragma unroll
      for (int m = 0; m < MI; ++m) slot[m] = 0;
    } else {
#pragma unroll
      for (int m = 0; m < MI; ++m) {
        if (!act[m]) continue;
        slot[m] = table_slot(q, sm, gid[m]);
        if (slot[m] >= 0) {
          atomicAdd(scount(q, sm, slot[m]), len[m]);
        } else {
          const long long g = gindex(q, gid[m]);
          if (g < 0) {
            act[m] = false;
            continue;
          }
          gi[m] = (uint32_t)g;
          atomicAdd(gword(q, 0, gi[m]), (unsigned long long)len[m]);
        }
      }
    }
    // ---- aggregates
    int last_col = -1;
    long long val[MI];
#pragma unroll
    for (int m = 0; m < MI; ++m) val[m] = 0;
    for (int ai = 0; ai < q.n_aggs; ++ai) {
      const AggDesc& a = q.aggs[ai];
      if (a.kind == AK_COUNT) continue;
      const ColDesc& c = q.cols[a.col];
      if (a.kind == AK_ISUM || a.kind == AK_ISUM2 || a.kind == AK_IMIN || a.kind == AK_IMAX) {
        // index column: only listed rows differ from the default, which the
        // finalize step adds back from COUNT
#pragma unroll
        for (int m = 0; m < MI; ++m) {
          long long v;
          if (act[m] && index_lookup(c, t, o[m], &v)) {
            if (a.kind == AK_ISUM) {
              sum_add(q, sm, a, slot[m], gi[m], index_delta(v, a.base));
            } else if (a.kind == AK_ISUM2) {
              const long long dv = v - a.base;   // |v - default| < 2^31 (planner)
              sum_add(q, sm, a, slot[m], gi[m], sext(dv * dv));
            } else {
              minmax_add(q, sm, a, slot[m], gi[m], v, a.kind == AK_IMIN);
              if (slot[m] >= 0) atomicAdd(slisted(q, sm, a, slot[m]), 1u);
              else atomicAdd(gword(q, a.gw + 1, gi[m]), 1ull);
            }
          }
        }
        continue;
      }
      if (a.expr != EXPR_NONE) {
        // position-wise arithmetic on two columns (Section 6), in actual values
        long long y[MI];
        auto read = [&](const ColDesc& cc, long long* out) {
          dispatch_col<SEG>(cc.enc, [&](auto et) {
            constexpr int E = decltype(et)::value;
#pragma unroll
            for (int m = 0; m < MI; ++m) out[m] = col_raw<E>(cc, t, o[m]) + (cc.raw_is_offset ? cc.base : 0);
          });
        };
        read(c, val);
        read(q.cols[a.col2], y);
#pragma unroll
        for (int m = 0; m < MI; ++m) val[m] = expr_apply(a.expr, val[m], y[m]);
        last_col = -1;
      } else if (a.col != last_col) {
        dispatch_col<SEG>(c.enc, [&](auto et) {
          constexpr int E = decltype(et)::value;
          if (a.n32) {
#pragma unroll
            for (int m = 0; m < MI; ++m) val[m] = (long long)col_raw32<E>(c, t, o[m]);
          } else {
#pragma unroll
            for (int m = 0; m < MI; ++m) val[m] = col_raw<E>(c, t, o[m]);
          }
        });
        last_col = a.col;
      }
      if (one_group && !SEG && (a.kind == AK_SUM ? a.red32 : a.w32)) {
        // warp reduction of the whole batch, one shared update
        int r;
        if (a.kind == AK_SUM) {
          int x = 0;
#pragma unroll
          for (int m = 0; m < MI; ++m) x += act[m] ? (int)val[m] : 0;
          r = __reduce_add_sync(0xFFFFFFFFu, x);
          if (lane == 0) {
            if (a.s32 == 3) split_add(sword32(q, sm, a.sw32, 0), sword32(q, sm, a.sw32 + 1, 0), (unsigned)r);
            else if (a.s32) atomicAdd(reinterpret_cast<unsigned*>(sword32(q, sm, a.sw32, 0)), (unsigned)r);
            else smem_add64(sword(q, sm, a.sw, 0), (long long)r);
          }
        } else {
          const bool mn = a.kind == AK_MIN;
          int x = mn ? INT_MAX : INT_MIN;
#pragma unroll
          for (int m = 0; m < MI; ++m)
            if (act[m]) x = mn ? min(x, (int)val[m]) : max(x, (int)val[m]);
          r = mn ? __reduce_min_sync(0xFFFFFFFFu, x) : __reduce_max_sync(0xFFFFFFFFu, x);
          if (lane == 0) {
            if (mn) atomicMin(sword32(q, sm, a.sw32, 0), r);
            else atomicMax(sword32(q, sm, a.sw32, 0), r);
          }
        }
        continue;
      }
#pragma unroll
      for (int m = 0; m < MI; ++m)
        if (act[m]) agg_item<SEG>(q, sm, a, slot[m], gi[m], val[m], len[m]);
    }
  }
}

}  // namespace cq
