// cq_query.cu -- the fused compressed-domain query kernel and its helpers.
//
// One persistent kernel evaluates a filter -> group-by -> aggregate plan over
// a table's compressed columns without decompressing them (Sections 6-7 of
// the paper).  The table's rows are cut into tiles of `tile_rows` rows; each
// CTA walks a contiguous range of tiles:
//
//  * Alignment (Section 6, Algorithm 1 generalised to k columns).  For each
//    RLE column the run ends that fall inside the tile are set as bits of a
//    tile-long bitmap, and for each index column its listed positions.  The
//    run (or listed entry) covering tile row o is then a popcount rank, so
//    the common refinement of all columns' runs never has to be sorted or
//    materialised.  In segment mode (every referenced column RLE or index)
//    the OR of the bitmaps gives the aligned segments themselves and the
//    kernel works per segment, weighting SUM by run length and COUNT by
//    length (Section 7, aggregating phase).
//  * Row-level columns (bit-packed, dictionary codes, plain) are streamed
//    tile by tile into shared memory with 1-D bulk copies on the TMA engine,
//    `stages` tiles ahead, each stage completing on an mbarrier; fields are
//    unpacked from shared memory.
//  * Predicates (a conjunction) run first over every row / segment; each
//    warp compacts its passing items, then computes their dense group id and
//    updates a shared-memory group table (dense bins for small key domains,
//    open addressing otherwise) that is flushed into exact global
//    accumulators.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <type_traits>

#include "cq_device.cuh"
#include "cq_internal.h"

namespace cq {

// ------------------------------------------------------------------ smem layout
struct SmemLayout {
  uint32_t stage, mbar, tkeys, tacc, bm, pre, ubm, upre, seg, clist, cursor, flags, misc, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(const QueryDesc& q) {
  SmemLayout L;
  const uint32_t nwords = q.tile_rows / 32;
  uint32_t off = 0;
  L.stage = off;
  off += q.seg_mode ? 0u : q.stages * q.stage_bytes;
  off = align_up(off, 16);
  L.mbar = off;
  off += 8u * (q.seg_mode ? 0u : q.stages);
  off = align_up(off, 16);
  L.tkeys = off;
  off += q.table_dense ? 0u : 4u * q.table_slots;
  off = align_up(off, 16);
  L.tacc = off;
  off += 8u * q.n_sw * q.table_slots;
  L.bm = off;
  off += 4u * nwords * q.n_bitmaps;
  L.pre = off;
  off += 4u * (nwords + 1) * q.n_bitmaps;
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
  L.cursor = off;
  off += 8u * kMaxBitmapCols;
  L.flags = off;
  off += 4u * 2 * kMaxBitmapCols;
  L.misc = off;
  off += 4u * 8;
  L.total = align_up(off, 128);
  return L;
}

size_t query_kernel_smem(const QueryDesc& q) { return smem_layout(q).total; }

struct Smem {
  uint8_t* stage;
  uint64_t* mbar;
  uint32_t* tkeys;
  unsigned long long* tacc;
  uint32_t* bm;
  uint32_t* pre;
  uint32_t* ubm;
  uint32_t* upre;
  uint16_t* seg;
  uint16_t* clist;
  unsigned long long* cursor;
  int* flags;   // [0..kMaxBitmapCols) done, [kMaxBitmapCols..) run ends exactly at the tile end
  int* misc;    // 0 occupancy, 1 rows since flush, 2 n segments
};

extern __shared__ __align__(128) uint8_t g_smem[];

__device__ __forceinline__ Smem carve(const QueryDesc& q) {
  const SmemLayout L = smem_layout(q);
  Smem s;
  s.stage = g_smem + L.stage;
  s.mbar = reinterpret_cast<uint64_t*>(g_smem + L.mbar);
  s.tkeys = reinterpret_cast<uint32_t*>(g_smem + L.tkeys);
  s.tacc = reinterpret_cast<unsigned long long*>(g_smem + L.tacc);
  s.bm = reinterpret_cast<uint32_t*>(g_smem + L.bm);
  s.pre = reinterpret_cast<uint32_t*>(g_smem + L.pre);
  s.ubm = reinterpret_cast<uint32_t*>(g_smem + L.ubm);
  s.upre = reinterpret_cast<uint32_t*>(g_smem + L.upre);
  s.seg = reinterpret_cast<uint16_t*>(g_smem + L.seg);
  s.clist = reinterpret_cast<uint16_t*>(g_smem + L.clist);
  s.cursor = reinterpret_cast<unsigned long long*>(g_smem + L.cursor);
  s.flags = reinterpret_cast<int*>(g_smem + L.flags);
  s.misc = reinterpret_cast<int*>(g_smem + L.misc);
  return s;
}

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

// Per-tile state needed to read a column at tile-relative row / segment start o.
struct TileCtx {
  const uint8_t* stage;   // current stage (row mode)
  uint32_t nwords;
};

// Raw value of column c at tile row o (see PredKind for "raw").
template <int ENC>
__device__ __forceinline__ long long col_raw(const ColDesc& c, const Smem& sm, const TileCtx& t, uint32_t o) {
  if constexpr (ENC == ENC_PLAIN) {
    const uint8_t* p = t.stage + c.stage_off;
    return c.v64 ? reinterpret_cast<const long long*>(p)[o] : (long long)reinterpret_cast<const int*>(p)[o];
  } else if constexpr (ENC == ENC_PACKED || ENC == ENC_DICT) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(t.stage + c.stage_off);
    const uint64_t f = extract_field(w, o, c.bw);
    return c.raw_is_offset ? (long long)f : (long long)(f + (uint64_t)c.base);
  } else if constexpr (ENC == ENC_RLE) {
    const uint32_t* B = sm.bm + c.bslot * t.nwords;
    const uint32_t* P = sm.pre + c.bslot * (t.nwords + 1);
    const uint64_t idx = sm.cursor[c.bslot] + rank_incl(B, P, o);
    return ldg_val(c.vals, idx, c.v64);
  } else {  // ENC_INDEX
    const uint32_t* B = sm.bm + c.bslot * t.nwords;
    const uint32_t wv = B[o >> 5];
    if (!((wv >> (o & 31)) & 1u)) return c.base;
    const uint32_t* P = sm.pre + c.bslot * (t.nwords + 1);
    const uint64_t idx = sm.cursor[c.bslot] + P[o >> 5] + __popc(wv & ((1u << (o & 31)) - 1u));
    return ldg_val(c.vals, idx, c.v64);
  }
}

// Index column at o: listed? and value.
__device__ __forceinline__ bool index_lookup(const ColDesc& c, const Smem& sm, const TileCtx& t, uint32_t o,
                                             long long* v) {
  const uint32_t* B = sm.bm + c.bslot * t.nwords;
  const uint32_t wv = B[o >> 5];
  if (!((wv >> (o & 31)) & 1u)) return false;
  const uint32_t* P = sm.pre + c.bslot * (t.nwords + 1);
  *v = ldg_val(c.vals, sm.cursor[c.bslot] + P[o >> 5] + __popc(wv & ((1u << (o & 31)) - 1u)), c.v64);
  return true;
}

__device__ __forceinline__ bool pred_eval(const QueryDesc& q, const PredDesc& p, long long v) {
  switch (p.kind) {
    case PK_RANGE: return v >= p.lo && v <= p.hi;
    case PK_NE: return v != p.lo;
    case PK_BITMAP: {
      if (v < p.lo || v > p.hi) return false;
      const unsigned long long d = (unsigned long long)(v - p.lo);
      return (__ldg(q.aux + p.aux_off + (uint32_t)(d >> 5)) >> (d & 31)) & 1u;
    }
    case PK_LIST: {
      const long long* L = reinterpret_cast<const long long*>(q.aux + p.aux_off);
      uint32_t lo = 0, hi = p.aux_len;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(L + mid) < v) lo = mid + 1; else hi = mid;
      }
      return lo < p.aux_len && __ldg(L + lo) == v;
    }
    case PK_FALSE: return false;
    default: return true;
  }
}

// digit of key k for raw value v; returns false when v is outside the domain
__device__ __forceinline__ bool key_digit(const QueryDesc& q, const KeyDesc& k, long long v, uint32_t* digit) {
  const unsigned long long d = (unsigned long long)(v - k.kmin);
  if (!k.remap) {
    if (v < k.kmin || d >= k.card) return false;
    *digit = (uint32_t)d;
    return true;
  }
  if (v < k.kmin || d >= 32ull * k.aux_len) return false;
  const uint32_t w = __ldg(q.aux + k.aux_off + (uint32_t)(d >> 5));
  if (!((w >> (d & 31)) & 1u)) return false;
  *digit = __ldg(q.aux + k.prefix_off + (uint32_t)(d >> 5)) + __popc(w & ((1u << (d & 31)) - 1u));
  return true;
}

// ------------------------------------------------------------------ group table
// multiplicative hashing: the top bits of gid * golden ratio select the slot
__device__ __forceinline__ uint32_t hash_gid(uint32_t g, uint32_t log2_slots) {
  return (g * 0x9E3779B1u) >> (32 - log2_slots);
}

// Shared-memory slot of gid, or -1 when the probe limit is hit (caller then
// updates the global accumulators directly).
__device__ __forceinline__ int table_slot(const QueryDesc& q, const Smem& sm, uint32_t gid) {
  if (q.table_dense) return (int)gid;
  const uint32_t mask = q.table_slots - 1;
  uint32_t h = hash_gid(gid, 31 - __clz(q.table_slots)) & mask;
  for (int probe = 0; probe < 32; ++probe) {
    uint32_t k = sm.tkeys[h];
    if (k == gid) return (int)h;
    if (k == kEmptyKey) {
      k = atomicCAS(&sm.tkeys[h], kEmptyKey, gid);
      if (k == kEmptyKey) {
        atomicAdd(&sm.misc[0], 1);
        return (int)h;
      }
      if (k == gid) return (int)h;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

__device__ __forceinline__ unsigned long long* gword(const QueryDesc& q, uint32_t w, uint32_t gid) {
  return q.gacc + (size_t)w * q.n_groups + gid;
}

// Apply one item (value v of aggregate a, weight len) to shared slot or global gid.
__device__ __forceinline__ void agg_update(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot,
                                           uint32_t gid, long long v, uint32_t len) {
  const uint32_t S = q.table_slots;
  switch (a.kind) {
    case AK_SUM:
    case AK_ISUM: {
      if (slot >= 0) {
        if (!a.wide) {
          const long long x = len == 1 ? v : v * (long long)len;
          atomicAdd(&sm.tacc[(size_t)a.sw * S + slot], (unsigned long long)x);
        } else {
          atomic_add_i128(&sm.tacc[(size_t)a.sw * S + slot], &sm.tacc[(size_t)(a.sw + 1) * S + slot],
                          len == 1 ? sext(v) : mul_s64(v, (long long)len));
        }
      } else {
        global_add_limbs(gword(q, a.gw, gid), gword(q, a.gw + 1, gid), gword(q, a.gw + 2, gid),
                         len == 1 ? sext(v) : mul_s64(v, (long long)len));
      }
      break;
    }
    case AK_MIN:
    case AK_IMIN:
      if (slot >= 0) atomicMin(reinterpret_cast<long long*>(&sm.tacc[(size_t)a.sw * S + slot]), v);
      else atomicMin(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
      break;
    case AK_MAX:
    case AK_IMAX:
      if (slot >= 0) atomicMax(reinterpret_cast<long long*>(&sm.tacc[(size_t)a.sw * S + slot]), v);
      else atomicMax(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
      break;
    default:
      break;
  }
  if (a.kind == AK_IMIN || a.kind == AK_IMAX) {   // listed count
    if (slot >= 0) atomicAdd(&sm.tacc[(size_t)(a.sw + 1) * S + slot], (unsigned long long)len);
    else atomicAdd(gword(q, a.gw + 1, gid), (unsigned long long)len);
  }
}

// Index column SUM: add (value - default) of a listed passing row (listed
// rows are single-row items, so the weight is 1).
__device__ __forceinline__ void isum_update(const QueryDesc& q, const Smem& sm, const AggDesc& a, int slot,
                                            uint32_t gid, long long v) {
  I128 x;
  x.lo = (unsigned long long)v - (unsigned long long)a.base;
  // borrow-aware high word of sext(v) - sext(base)
  x.hi = (v < 0 ? -1ll : 0ll) - (a.base < 0 ? -1ll : 0ll) - ((unsigned long long)v < (unsigned long long)a.base ? 1ll : 0ll);
  const uint32_t S = q.table_slots;
  if (slot >= 0) {
    if (!a.wide) atomicAdd(&sm.tacc[(size_t)a.sw * S + slot], x.lo);
    else atomic_add_i128(&sm.tacc[(size_t)a.sw * S + slot], &sm.tacc[(size_t)(a.sw + 1) * S + slot], x);
  } else {
    global_add_limbs(gword(q, a.gw, gid), gword(q, a.gw + 1, gid), gword(q, a.gw + 2, gid), x);
  }
}

__device__ __forceinline__ void reset_slot(const QueryDesc& q, const Smem& sm, uint32_t s) {
  const uint32_t S = q.table_slots;
  sm.tacc[s] = 0;
  for (int i = 0; i < q.n_aggs; ++i) {
    const AggDesc& a = q.aggs[i];
    switch (a.kind) {
      case AK_SUM:
      case AK_ISUM:
        sm.tacc[(size_t)a.sw * S + s] = 0;
        if (a.wide) sm.tacc[(size_t)(a.sw + 1) * S + s] = 0;
        break;
      case AK_MIN:
      case AK_IMIN:
        sm.tacc[(size_t)a.sw * S + s] = (unsigned long long)LLONG_MAX;
        if (a.kind == AK_IMIN) sm.tacc[(size_t)(a.sw + 1) * S + s] = 0;
        break;
      case AK_MAX:
      case AK_IMAX:
        sm.tacc[(size_t)a.sw * S + s] = (unsigned long long)LLONG_MIN;
        if (a.kind == AK_IMAX) sm.tacc[(size_t)(a.sw + 1) * S + s] = 0;
        break;
      default:
        break;
    }
  }
  if (!q.table_dense) sm.tkeys[s] = kEmptyKey;
}

// Add every occupied slot into the global accumulators and clear the table.
__device__ void flush_table(const QueryDesc& q, const Smem& sm) {
  const uint32_t S = q.table_slots;
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
    const unsigned long long cnt = sm.tacc[s];
    if (cnt == 0) {
      if (!q.table_dense) sm.tkeys[s] = kEmptyKey;
      continue;
    }
    const uint32_t gid = q.table_dense ? s : sm.tkeys[s];
    atomicAdd(gword(q, 0, gid), cnt);
    for (int i = 0; i < q.n_aggs; ++i) {
      const AggDesc& a = q.aggs[i];
      switch (a.kind) {
        case AK_SUM:
        case AK_ISUM: {
          I128 x;
          if (a.wide) {
            x.lo = sm.tacc[(size_t)a.sw * S + s];
            x.hi = (long long)sm.tacc[(size_t)(a.sw + 1) * S + s];
          } else {
            x = sext((long long)sm.tacc[(size_t)a.sw * S + s]);
          }
          global_add_limbs(gword(q, a.gw, gid), gword(q, a.gw + 1, gid), gword(q, a.gw + 2, gid), x);
          break;
        }
        case AK_MIN:
        case AK_IMIN: {
          const long long v = (long long)sm.tacc[(size_t)a.sw * S + s];
          if (v != LLONG_MAX) atomicMin(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
          break;
        }
        case AK_MAX:
        case AK_IMAX: {
          const long long v = (long long)sm.tacc[(size_t)a.sw * S + s];
          if (v != LLONG_MIN) atomicMax(reinterpret_cast<long long*>(gword(q, a.gw, gid)), v);
          break;
        }
        default:
          break;
      }
      if (a.kind == AK_IMIN || a.kind == AK_IMAX) {
        const unsigned long long lc = sm.tacc[(size_t)(a.sw + 1) * S + s];
        if (lc) atomicAdd(gword(q, a.gw + 1, gid), lc);
      }
    }
    reset_slot(q, sm, s);
  }
}

// ------------------------------------------------------------------ tile alignment
// Build the per-tile bitmaps of every RLE / index column for rows [s, e) and
// their word prefix popcounts.  RLE: bit o set when a run ends at row s + o
// (exclusive end), i.e. row s + o starts a new run.  Index: bit o set when
// row s + o is listed.  Column j's cursor must hold the first run with end
// > s (RLE) / the first position >= s (index).
__device__ void build_bitmaps(const QueryDesc& q, const Smem& sm, unsigned long long s, unsigned long long e,
                              uint32_t nwords) {
  const int nb = q.n_bitmaps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < nwords * nb; i += blockDim.x) sm.bm[i] = 0;
  if (threadIdx.x < 2 * kMaxBitmapCols) sm.flags[threadIdx.x] = 0;
  __syncthreads();
  if (nb > 0) {
    // warps are dealt to columns round-robin; warp w serves column w % nb
    const int j = warp % nb;
    const int gi = warp / nb;
    const int G = (kWarps - j + nb - 1) / nb;
    const ColDesc* cd = nullptr;
    for (int c = 0; c < q.n_cols; ++c)
      if (q.cols[c].bslot == j) cd = &q.cols[c];
    const bool is_rle = cd->enc == ENC_RLE;
    const unsigned long long cur = sm.cursor[j];
    uint32_t* B = sm.bm + j * nwords;
    for (int it = 0;; ++it) {
      const int col_done = __shfl_sync(0xFFFFFFFFu, sm.flags[j], 0);
      if (!col_done) {
        const unsigned long long idx = cur + ((unsigned long long)it * G + gi) * 32 + lane;
        bool stop = false;
        if (idx < cd->n) {
          const long long x = ldg_val(cd->ends, idx, cd->e64);
          if ((unsigned long long)x < e) {
            // a boundary before the tile would mean a corrupt cursor: flag it, never write
            if ((unsigned long long)x < s || (is_rle && (unsigned long long)x == s)) {
              atomicCAS(q.err, 0, (int)CQ_ERR_INVALID_ARG);
            } else {
              const uint32_t o = (uint32_t)((unsigned long long)x - s);
              atomicOr(&B[o >> 5], 1u << (o & 31));
            }
          } else {
            stop = true;
            if (is_rle && (unsigned long long)x == e) sm.flags[kMaxBitmapCols + j] = 1;
          }
        } else {
          stop = true;
        }
        if (__any_sync(0xFFFFFFFFu, stop) && lane == 0) sm.flags[j] = 1;
      }
      __syncthreads();
      bool all = true;
      for (int c = 0; c < nb; ++c) all = all && sm.flags[c];
      __syncthreads();
      if (all) break;
    }
    // word prefix popcounts, one warp per column
    for (int c = warp; c < nb; c += kWarps) {
      const uint32_t* Bc = sm.bm + c * nwords;
      uint32_t* Pc = sm.pre + c * (nwords + 1);
      const uint32_t per = (nwords + 31) / 32;
      uint32_t local = 0;
      for (uint32_t k = 0; k < per; ++k) {
        const uint32_t w = lane * per + k;
        if (w < nwords) local += __popc(Bc[w]);
      }
      uint32_t incl = local;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
      }
      uint32_t run = incl - local;
      for (uint32_t k = 0; k < per; ++k) {
        const uint32_t w = lane * per + k;
        if (w < nwords) {
          Pc[w] = run;
          run += __popc(Bc[w]);
        }
      }
      if (lane == 31) Pc[nwords] = incl;
    }
  }
  __syncthreads();
}

// Segment mode: union of all bitmaps -> segment start list in sm.seg.
// Index columns split the tile before and after every listed row.
__device__ void build_segments(const QueryDesc& q, const Smem& sm, uint32_t nwords, uint32_t rows) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) {
    uint32_t u = 0;
    for (int c = 0; c < q.n_cols; ++c) {
      const ColDesc& cd = q.cols[c];
      if (cd.bslot == 0xFF) continue;
      const uint32_t* B = sm.bm + cd.bslot * nwords;
      if (cd.enc == ENC_RLE) {
        u |= B[w];
      } else {
        const uint32_t prev = w ? B[w - 1] : 0u;
        u |= B[w] | (B[w] << 1) | (prev >> 31);
      }
    }
    if (w == 0) u &= ~1u;   // row 0 always starts a segment
    if (w == (rows >> 5) && (rows & 31)) u &= (1u << (rows & 31)) - 1u;
    if (w > (rows >> 5) || (w == (rows >> 5) && !(rows & 31))) u = 0;
    sm.ubm[w] = u;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t per = (nwords + 31) / 32;
    uint32_t local = 0;
    for (uint32_t k = 0; k < per; ++k) {
      const uint32_t w = lane * per + k;
      if (w < nwords) local += __popc(sm.ubm[w]);
    }
    uint32_t incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t run = incl - local;
    for (uint32_t k = 0; k < per; ++k) {
      const uint32_t w = lane * per + k;
      if (w < nwords) {
        sm.upre[w] = run;
        run += __popc(sm.ubm[w]);
      }
    }
    if (lane == 31) {
      sm.misc[2] = (int)(incl + 1);
      sm.seg[0] = 0;
      sm.seg[incl + 1] = (uint16_t)rows;
    }
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) {
    uint32_t u = sm.ubm[w];
    uint32_t k = 1 + sm.upre[w];
    while (u) {
      const int b = __ffs(u) - 1;
      sm.seg[k++] = (uint16_t)(w * 32 + b);
      u &= u - 1;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ the kernel
template <bool SEG>
__global__ void __launch_bounds__(kThreads, 1) fused_query_kernel(const __grid_constant__ QueryDesc q) {
  const Smem sm = carve(q);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t T = q.tile_rows;
  const uint32_t nwords = T / 32;
  const unsigned long long t_begin = (unsigned long long)blockIdx.x * q.n_tiles / gridDim.x;
  const unsigned long long t_end = (unsigned long long)(blockIdx.x + 1) * q.n_tiles / gridDim.x;
  if (t_begin >= t_end) return;

  // ---- init shared group table, barriers, cursors
  for (uint32_t sl = threadIdx.x; sl < q.table_slots; sl += blockDim.x) reset_slot(q, sm, sl);
  if (threadIdx.x < 8) sm.misc[threadIdx.x] = 0;
  if (!SEG && threadIdx.x == 0) {
    for (int st = 0; st < q.stages; ++st) mbar_init(&sm.mbar[st], 1);
    fence_barrier_init();
  }
  if (warp < q.n_bitmaps) {
    const ColDesc* cd = nullptr;
    for (int c = 0; c < q.n_cols; ++c)
      if (q.cols[c].bslot == warp) cd = &q.cols[c];
    const long long s0 = (long long)(t_begin * T);
    // RLE: first run whose exclusive end exceeds s0; index: first position >= s0
    const unsigned long long cur =
        warp_count_below(cd->ends, cd->e64, cd->n, s0, /*strict=*/cd->enc == ENC_INDEX);
    if (lane == 0) sm.cursor[warp] = cur;
  }
  __syncthreads();

  // ---- bulk-copy producer (thread 0): tile u -> stage (u - t_begin) % stages
  auto issue = [&](unsigned long long u) {
    const uint32_t st = (uint32_t)((u - t_begin) % q.stages);
    uint8_t* dst = sm.stage + (size_t)st * q.stage_bytes;
    const unsigned long long r0 = u * T;
    const unsigned long long rows = (q.n_rows - r0) < (unsigned long long)T ? (q.n_rows - r0) : (unsigned long long)T;
    uint32_t total = 0;
    uint32_t bytes[kMaxCols];
    for (int i = 0; i < q.n_row_cols; ++i) {
      const ColDesc& c = q.cols[q.row_cols[i]];
      const uint32_t bits = c.enc == ENC_PLAIN ? (c.v64 ? 64u : 32u) : (uint32_t)c.bw;
      bytes[i] = (uint32_t)(((rows * bits + 7) / 8 + 15) / 16 * 16);
      total += bytes[i];
    }
    mbar_arrive_expect_tx(&sm.mbar[st], total);
    for (int i = 0; i < q.n_row_cols; ++i) {
      const ColDesc& c = q.cols[q.row_cols[i]];
      const uint32_t bits = c.enc == ENC_PLAIN ? (c.v64 ? 64u : 32u) : (uint32_t)c.bw;
      const uint8_t* src = reinterpret_cast<const uint8_t*>(c.vals) + r0 * bits / 8;
      bulk_g2s(dst + c.stage_off, src, bytes[i], &sm.mbar[st]);
    }
  };
  if (!SEG && threadIdx.x == 0) {
    for (unsigned long long u = t_begin; u < t_end && u < t_begin + q.stages - 1; ++u) issue(u);
  }

  for (unsigned long long t = t_begin; t < t_end; ++t) {
    const unsigned long long s = t * T;
    const unsigned long long e = (s + T < q.n_rows) ? s + T : q.n_rows;
    const uint32_t rows = (uint32_t)(e - s);
    if (!SEG && threadIdx.x == 0 && t + q.stages - 1 < t_end) issue(t + q.stages - 1);

    build_bitmaps(q, sm, s, e, nwords);
    if (SEG) build_segments(q, sm, nwords, rows);

    TileCtx tc;
    tc.nwords = nwords;
    tc.stage = sm.stage;
    if (!SEG) {
      const uint32_t st = (uint32_t)((t - t_begin) % q.stages);
      const uint32_t parity = (uint32_t)(((t - t_begin) / q.stages) & 1ull);
      tc.stage = sm.stage + (size_t)st * q.stage_bytes;
      mbar_wait_bounded(&sm.mbar[st], parity, q.err);
    }

    // ---- phase P: predicates over this warp's items, compact the passing ones
    const uint32_t n_items = SEG ? (uint32_t)sm.misc[2] : rows;
    const uint32_t per_warp = ((n_items + kWarps * 32 - 1) / (kWarps * 32)) * 32;
    const uint32_t first = warp * per_warp;
    const int groups = (int)(per_warp / 32);
    uint32_t item[kMaxGroupsPerWarp];
    bool ok[kMaxGroupsPerWarp];
#pragma unroll
    for (int g = 0; g < kMaxGroupsPerWarp; ++g) {
      const uint32_t it = first + g * 32 + lane;
      ok[g] = g < groups && it < n_items;
      item[g] = it;
    }
    for (int pi = 0; pi < q.n_preds; ++pi) {
      const PredDesc& p = q.preds[pi];
      const ColDesc& c = q.cols[p.col];
      dispatch_enc(c.enc, [&](auto tag) {
        constexpr int E = decltype(tag)::value;
#pragma unroll
        for (int g = 0; g < kMaxGroupsPerWarp; ++g) {
          if (ok[g]) {
            const uint32_t o = SEG ? (uint32_t)sm.seg[item[g]] : item[g];
            ok[g] = pred_eval(q, p, col_raw<E>(c, sm, tc, o));
          }
        }
      });
    }
    uint16_t* mylist = sm.clist + warp * (T / kWarps);
    uint32_t n_pass = 0;
#pragma unroll
    for (int g = 0; g < kMaxGroupsPerWarp; ++g) {
      if (g < groups) {
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok[g]);
        if (ok[g]) mylist[n_pass + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)item[g];
        n_pass += __popc(bal);
      }
    }
    __syncwarp();

    // ---- phase A: group id, slot, aggregate updates for the passing items
    for (uint32_t base = 0; base < n_pass; base += 32 * kMaxGroupsPerWarp) {
      uint32_t gid[kMaxGroupsPerWarp];
      uint32_t off[kMaxGroupsPerWarp];
      uint32_t len[kMaxGroupsPerWarp];
      bool act[kMaxGroupsPerWarp];
      bool bad[kMaxGroupsPerWarp];
#pragma unroll
      for (int m = 0; m < kMaxGroupsPerWarp; ++m) {
        const uint32_t j = base + m * 32 + lane;
        act[m] = j < n_pass;
        bad[m] = false;
        gid[m] = 0;
        off[m] = 0;
        len[m] = 1;
        if (act[m]) {
          const uint32_t itm = mylist[j];
          if (SEG) {
            off[m] = sm.seg[itm];
            len[m] = (uint32_t)sm.seg[itm + 1] - off[m];
          } else {
            off[m] = itm;
          }
        }
      }
      for (int ki = 0; ki < q.n_keys; ++ki) {
        const KeyDesc& k = q.keys[ki];
        const ColDesc& c = q.cols[k.col];
        dispatch_enc(c.enc, [&](auto tag) {
          constexpr int E = decltype(tag)::value;
#pragma unroll
          for (int m = 0; m < kMaxGroupsPerWarp; ++m) {
            if (act[m]) {
              uint32_t d;
              if (key_digit(q, k, col_raw<E>(c, sm, tc, off[m]), &d)) gid[m] += d * (uint32_t)k.stride;
              else bad[m] = true;
            }
          }
        });
      }
      int slot[kMaxGroupsPerWarp];
#pragma unroll
      for (int m = 0; m < kMaxGroupsPerWarp; ++m) {
        slot[m] = -1;
        if (act[m] && bad[m]) {
          atomicCAS(q.err, 0, (int)CQ_ERR_INVALID_ARG);
          act[m] = false;
        }
        if (act[m]) {
          slot[m] = table_slot(q, sm, gid[m]);
          if (slot[m] >= 0) atomicAdd(&sm.tacc[slot[m]], (unsigned long long)len[m]);
          else atomicAdd(gword(q, 0, gid[m]), (unsigned long long)len[m]);
        }
      }
      for (int ai = 0; ai < q.n_aggs; ++ai) {
        const AggDesc& a = q.aggs[ai];
        if (a.kind == AK_COUNT) continue;
        const ColDesc& c = q.cols[a.col];
        if (a.kind == AK_ISUM || a.kind == AK_IMIN || a.kind == AK_IMAX) {
#pragma unroll
          for (int m = 0; m < kMaxGroupsPerWarp; ++m) {
            long long v;
            if (act[m] && index_lookup(c, sm, tc, off[m], &v)) {
              if (a.kind == AK_ISUM) isum_update(q, sm, a, slot[m], gid[m], v);
              else agg_update(q, sm, a, slot[m], gid[m], v, len[m]);
            }
          }
          continue;
        }
        dispatch_enc(c.enc, [&](auto tag) {
          constexpr int E = decltype(tag)::value;
#pragma unroll
          for (int m = 0; m < kMaxGroupsPerWarp; ++m) {
            if (act[m]) agg_update(q, sm, a, slot[m], gid[m], col_raw<E>(c, sm, tc, off[m]), len[m]);
          }
        });
      }
    }
    __syncthreads();

    // ---- advance cursors, flush the table when needed
    if (threadIdx.x < q.n_bitmaps) {
      const int j = threadIdx.x;
      const uint32_t* P = sm.pre + j * (nwords + 1);
      sm.cursor[j] += P[nwords] + (unsigned long long)sm.flags[kMaxBitmapCols + j];
    }
    if (threadIdx.x == 0) sm.misc[1] += (int)rows;
    __syncthreads();
    const bool last = (t + 1 == t_end);
    const bool need = last || (!q.table_dense && sm.misc[0] * 2 > (int)q.table_slots) ||
                      (unsigned)sm.misc[1] + T > q.flush_rows;
    if (need) {
      flush_table(q, sm);
      __syncthreads();
      if (threadIdx.x == 0) {
        sm.misc[0] = 0;
        sm.misc[1] = 0;
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ init / finalize
__global__ void init_global_kernel(const __grid_constant__ QueryDesc q) {
  const size_t G = q.n_groups;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G; i += (size_t)gridDim.x * blockDim.x) {
    q.gacc[i] = 0;
    for (int ai = 0; ai < q.n_aggs; ++ai) {
      const AggDesc& a = q.aggs[ai];
      switch (a.kind) {
        case AK_SUM:
        case AK_ISUM:
          q.gacc[(size_t)a.gw * G + i] = 0;
          q.gacc[(size_t)(a.gw + 1) * G + i] = 0;
          q.gacc[(size_t)(a.gw + 2) * G + i] = 0;
          break;
        case AK_MIN:
        case AK_IMIN:
          q.gacc[(size_t)a.gw * G + i] = (unsigned long long)LLONG_MAX;
          if (a.kind == AK_IMIN) q.gacc[(size_t)(a.gw + 1) * G + i] = 0;
          break;
        case AK_MAX:
        case AK_IMAX:
          q.gacc[(size_t)a.gw * G + i] = (unsigned long long)LLONG_MIN;
          if (a.kind == AK_IMAX) q.gacc[(size_t)(a.gw + 1) * G + i] = 0;
          break;
        default:
          break;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *q.err = 0;
    *q.out_count = 0;
  }
}

constexpr int kFinBlock = 1024;

__device__ __forceinline__ bool group_present(const QueryDesc& q, size_t g) {
  return q.gacc[g] != 0 || (q.n_keys == 0 && g == 0);
}

__global__ void finalize_count_kernel(const __grid_constant__ QueryDesc q) {
  const size_t g = blockIdx.x * (size_t)kFinBlock + threadIdx.x;
  const bool p = g < q.n_groups && group_present(q, g);
  const int c = __syncthreads_count(p);
  if (threadIdx.x == 0) q.block_counts[blockIdx.x] = (unsigned)c;
}

__global__ void finalize_scan_kernel(const __grid_constant__ QueryDesc q, unsigned n_blocks) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned base = 0; base < n_blocks; base += blockDim.x) {
    const unsigned i = base + threadIdx.x;
    const unsigned v = i < n_blocks ? q.block_counts[i] : 0u;
    unsigned incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned x = lane < (int)(blockDim.x / 32) ? warp_tot[lane] : 0u;
      unsigned wi = x;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
        if (lane >= d) wi += y;
      }
      warp_tot[lane] = wi - x;
    }
    __syncthreads();
    const unsigned long long c0 = carry;
    if (i < n_blocks) q.block_counts[i] = (unsigned)(c0 + warp_tot[warp] + incl - v);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_tot[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *q.out_count = carry;
}

__device__ __forceinline__ I128 read_sum(const QueryDesc& q, uint32_t gw, size_t g) {
  const size_t G = q.n_groups;
  const unsigned long long w0 = q.gacc[(size_t)gw * G + g];
  const unsigned long long w1 = q.gacc[(size_t)(gw + 1) * G + g];
  const long long w2 = (long long)q.gacc[(size_t)(gw + 2) * G + g];
  // value = w0 + w1 * 2^32 + w2 * 2^64
  I128 r;
  const unsigned long long a = w0 + (w1 << 32);
  const unsigned long long c1 = a < w0 ? 1ull : 0ull;
  r.lo = a;
  r.hi = w2 + (long long)(w1 >> 32) + (long long)c1;
  return r;
}

__device__ __forceinline__ I128 add128(I128 a, I128 b) {
  I128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}

__global__ void finalize_write_kernel(const __grid_constant__ QueryDesc q) {
  __shared__ unsigned warp_cnt[kFinBlock / 32];
  const size_t g = blockIdx.x * (size_t)kFinBlock + threadIdx.x;
  const bool p = g < q.n_groups && group_present(q, g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, p);
  if (lane == 0) warp_cnt[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    const unsigned x = warp_cnt[lane];
    unsigned incl = x;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    warp_cnt[lane] = incl - x;
  }
  __syncthreads();
  if (!p) return;
  const size_t row = q.block_counts[blockIdx.x] + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
  const unsigned long long cnt = q.gacc[g];
  for (uint32_t oc = 0; oc < q.n_out; ++oc) {
    const uint32_t idx = q.out_index[oc];
    if (q.out_is_key[oc]) {
      const KeyDesc& k = q.keys[idx];
      const uint32_t digit = (uint32_t)((g / k.stride) % k.card);
      long long raw;
      if (k.remap) {
        raw = reinterpret_cast<const long long*>(q.aux + k.list_off)[digit];
      } else {
        raw = k.kmin + (long long)digit;
      }
      const ColDesc& c = q.cols[k.col];
      const long long val = c.raw_is_offset && c.enc == ENC_PACKED ? (long long)((unsigned long long)raw + (unsigned long long)c.base) : raw;
      reinterpret_cast<long long*>(q.out[oc])[row] = val;
      continue;
    }
    const AggDesc& a = q.aggs[idx];
    switch (a.kind) {
      case AK_COUNT:
        reinterpret_cast<unsigned long long*>(q.out[oc])[row] = cnt;
        break;
      case AK_SUM:
      case AK_ISUM: {
        I128 x = read_sum(q, a.gw, g);
        if (a.base != 0) x = add128(x, mul_s64(a.base, (long long)cnt));   // base / default times COUNT
        if (a.op == CQ_AVG) {
          reinterpret_cast<double*>(q.out[oc])[row] = cnt ? i128_to_double(x) / __ull2double_rn(cnt) : 0.0;
        } else {
          const bool fits = (x.hi == 0 && (long long)x.lo >= 0) || (x.hi == -1 && (long long)x.lo < 0);
          if (!fits) atomicCAS(q.err, 0, (int)CQ_ERR_OVERFLOW);
          reinterpret_cast<long long*>(q.out[oc])[row] = (long long)x.lo;
        }
        break;
      }
      case AK_MIN:
      case AK_MAX: {
        long long v = (long long)q.gacc[(size_t)a.gw * q.n_groups + g];
        if (cnt == 0) v = 0;
        else v = (long long)((unsigned long long)v + (unsigned long long)a.base);
        reinterpret_cast<long long*>(q.out[oc])[row] = v;
        break;
      }
      case AK_IMIN:
      case AK_IMAX: {
        const long long lv = (long long)q.gacc[(size_t)a.gw * q.n_groups + g];
        const unsigned long long lc = q.gacc[(size_t)(a.gw + 1) * q.n_groups + g];
        long long v;
        if (cnt == 0) v = 0;
        else if (lc == 0) v = a.base;
        else if (lc < cnt) v = a.kind == AK_IMIN ? (lv < a.base ? lv : a.base) : (lv > a.base ? lv : a.base);
        else v = lv;
        reinterpret_cast<long long*>(q.out[oc])[row] = v;
        break;
      }
      default:
        break;
    }
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t query_kernel_set_smem(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(fused_query_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fused_query_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_init_global(const QueryDesc& q, cudaStream_t s) {
  const unsigned long long nblk = (q.n_groups + 255) / 256;
  const unsigned blocks = (unsigned)(nblk < 4096ull ? nblk : 4096ull);
  init_global_kernel<<<blocks ? blocks : 1, 256, 0, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_query(const QueryDesc& q, cudaStream_t s, int num_sms, int ctas_per_sm, uint32_t grid_ctas) {
  const unsigned long long want =
      grid_ctas ? (unsigned long long)grid_ctas : (unsigned long long)num_sms * (unsigned long long)ctas_per_sm;
  const unsigned grid = (unsigned)(q.n_tiles < want ? q.n_tiles : want);
  if (grid == 0) return cudaSuccess;
  if (q.seg_mode) fused_query_kernel<true><<<grid, kThreads, q.smem_bytes, s>>>(q);
  else fused_query_kernel<false><<<grid, kThreads, q.smem_bytes, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const QueryDesc& q, cudaStream_t s) {
  const unsigned nb = (unsigned)((q.n_groups + kFinBlock - 1) / kFinBlock);
  finalize_count_kernel<<<nb, kFinBlock, 0, s>>>(q);
  finalize_scan_kernel<<<1, 1024, 0, s>>>(q, nb);
  finalize_write_kernel<<<nb, kFinBlock, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace cq
