// cq_seg.cuh -- segment-mode steps of the fused query: per-tile alignment
// bitmaps, the aligned segment list, and the walk over a range of tiles.
// Used by the one-query kernel (cq_query.cu) and by the persistent batch
// kernel (cq_batch.cu).
//
// Alignment (Section 6, Algorithm 1 generalised to k columns): the run ends of
// every RLE column that fall in a tile are set as bits of a tile-long bitmap,
// the listed positions of every index column likewise, and the run (or listed
// entry) covering tile row o is a popcount rank.  The OR of the bitmaps gives
// the aligned segments; SUM adds value x run length and COUNT adds length
// (Section 7).
#pragma once

#include "cq_phases.cuh"

namespace cq {

// ------------------------------------------------------------------ tile alignment
// Build the per-tile bitmaps of every RLE / index column for rows [s, e) and
// their word prefix popcounts.  RLE: bit o set when a run ends at row s + o
// (exclusive end), i.e. row s + o starts a new run.  Index: bit o set when
// row s + o is listed.  Column j's cursor must hold the first run with end
// > s (RLE) / the first position >= s (index).
__device__ inline void build_bitmaps(const QueryDesc& q, const Smem& sm, unsigned long long s, unsigned long long e,
                              uint32_t nwords) {
  const int nb = q.n_bitmaps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < nwords * nb; i += blockDim.x) sm.bm[i] = 0;
  __syncthreads();
  if (nb > 0) {
    // warps are dealt to columns round-robin; warp w serves column w % nb
    // (a batch kernel's extra helper warp only joins the barriers)
    const bool active = warp < kWarps;
    const int j = warp % nb;
    const int gi = warp / nb;
    const int G = (kWarps - j + nb - 1) / nb;
    const ColDesc* cd = nullptr;
    for (int c = 0; c < q.n_cols; ++c)
      if (q.cols[c].bslot == j) cd = &q.cols[c];
    const bool is_rle = cd->enc == ENC_RLE;
    const unsigned long long cur = sm.tcur[j];
    uint32_t* B = sm.bm + j * nwords;
    // A column is done once an entry at or past the tile end was seen.  The
    // done flags are written only before the first barrier of an iteration
    // and read only between its two barriers, so every warp of a column
    // sees the same state: a warp must not skip its entries of an iteration
    // because another warp of the column stopped in that same iteration.
    bool col_done = false;
    for (int it = 0;; ++it) {
      if (active && !col_done) {
        const unsigned long long idx = cur + ((unsigned long long)it * G + gi) * 32 + lane;
        bool stop = false;
        if (idx < cd->n) {
          const long long x = ldg_val(cd->ends, idx, cd->e64);
          if ((unsigned long long)x < e) {
            // a boundary before the tile would mean a corrupt cursor: flag it, never write
            if ((unsigned long long)x < s || (is_rle && (unsigned long long)x == s)) {
              report(q, CQ_ERR_INVALID_ARG, 2ull + ((unsigned long long)j << 8), s, (unsigned long long)x);
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
      col_done = sm.flags[j] != 0;
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
__device__ inline void build_segments(const QueryDesc& q, const Smem& sm, uint32_t nwords, uint32_t rows) {
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

// Filter and aggregate one aligned segment of L rows starting at row s over
// which every column is constant: value(c) is column c's value there (an RLE
// column's run value, an index column's listed value or default), listed(c,
// &v) tells whether an index column lists the (single) row, with its value.
// COUNT += L, SUM += value x L, MIN / MAX on the value (Section 7); index
// aggregates take listed rows only (finalize adds the default from COUNT).
// One thread per segment.
template <class Value, class Listed>
__device__ inline void segment_update(const QueryDesc& q, const Smem& sm, const uint32_t* aux, unsigned long long s,
                                      unsigned long long L, Value value, Listed listed) {
  // the filter's clauses: a predicate alone must hold, a clause needs one
  // member that holds (pred_eval complements negated predicates)
  bool acc = false;
  for (int i = 0; i < q.n_preds; ++i) {
    const PredDesc& p = q.preds[i];
    if (p.clause == PC_ALONE) {
      if (!pred_eval(p, aux, value(p.col))) return;
    } else {
      acc = acc || pred_eval(p, aux, value(p.col));
      if (p.clause == PC_LAST) {
        if (!acc) return;
        acc = false;
      }
    }
  }
  unsigned long long gid = 0;
  for (int ki = 0; ki < q.n_keys; ++ki) {
    const KeyDesc& k = q.keys[ki];
    const long long v = value(k.col);
    unsigned long long d;
    if (!key_digit(k, aux, v, &d)) {
      report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)ki << 8), s, (unsigned long long)v);
      return;
    }
    gid += d * k.stride;
  }
  const int slot = q.n_groups == 1 && !q.ghash ? 0 : table_slot(q, sm, gid);
  uint32_t gi = 0;
  if (slot >= 0) {
    atomicAdd(scount(q, sm, slot), (unsigned)L);
  } else {
    const long long g = gindex(q, gid);
    if (g < 0) return;
    gi = (uint32_t)g;
    atomicAdd(gword(q, 0, gi), L);
  }
  // an aggregate's value on the segment: the column's, or the expression
  // of two columns' values (Section 6: arithmetic on aligned columns)
  auto aval = [&](const AggDesc& a) -> long long {
    const long long x = value(a.col);
    return a.expr == EXPR_NONE ? x : expr_apply(a.expr, x, value(a.col2));
  };
  for (int ai = 0; ai < q.n_aggs; ++ai) {
    const AggDesc& a = q.aggs[ai];
    if (a.kind == AK_SUM) {
      sum_add(q, sm, a, slot, gi, mul_s64(aval(a), (long long)L));
    } else if (a.kind == AK_SUM2) {
      const long long v = value(a.col);   // |v| < 2^31 (planner)
      sum_add(q, sm, a, slot, gi, mul_s64(v * v, (long long)L));
    } else if (a.kind == AK_MIN || a.kind == AK_MAX) {
      minmax_add(q, sm, a, slot, gi, aval(a), a.kind == AK_MIN);
    } else if (a.kind != AK_COUNT) {
      long long v;
      if (!listed(a.col, &v)) continue;
      if (a.kind == AK_ISUM) {
        sum_add(q, sm, a, slot, gi, index_delta(v, a.base));
      } else if (a.kind == AK_ISUM2) {
        const long long dv = v - a.base;
        sum_add(q, sm, a, slot, gi, sext(dv * dv));
      } else {
        minmax_add(q, sm, a, slot, gi, v, a.kind == AK_IMIN);
        if (slot >= 0) atomicAdd(slisted(q, sm, a, slot), 1u);
        else atomicAdd(gword(q, a.gw + 1, gi), 1ull);
      }
    }
  }
}

// A segment of L rows at row s inside which no column has a boundary: each
// RLE column holds the run at its cursor, each index column its default.
__device__ inline void seg_span_update(const QueryDesc& q, const Smem& sm, const uint32_t* aux, unsigned long long s,
                                       unsigned long long L) {
  auto value = [&](int c) -> long long {
    const ColDesc& cd = q.cols[c];
    if (cd.enc == ENC_RLE) return ldg_val(cd.vals, sm.tcur[cd.bslot], cd.v64);
    return cd.base;
  };
  auto listed = [&](int, long long*) { return false; };
  segment_update(q, sm, aux, s, L, value, listed);
}

// Walk tiles [t_begin, t_end) of one segment-mode query: reset the group
// table, then per tile build the bitmaps and segments, filter, aggregate,
// and flush the table when it fills and after the last tile.  kWarps warps
// do the work; further warps of the block (the batch kernel's helper warp)
// only take part in the block barriers.
template <int GPW>
__device__ __forceinline__ void seg_range(const QueryDesc& q, const Smem& sm, unsigned long long t_begin,
                                          unsigned long long t_end) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t T = q.tile_rows;
  const uint32_t nwords = T / 32;

  for (uint32_t sl = threadIdx.x; sl < q.table_slots; sl += blockDim.x) reset_slot(q, sm, sl);
  if (threadIdx.x < 8) sm.misc[threadIdx.x] = 0;
  if (threadIdx.x < 2 * kMaxBitmapCols) sm.flags[threadIdx.x] = 0;
  if (threadIdx.x < kMaxBitmapCols) sm.wcnt[threadIdx.x] = 0;
  const bool aux_smem = q.aux_words <= kAuxSmemWords;
  if (aux_smem)
    for (uint32_t i = threadIdx.x; i < q.aux_words; i += blockDim.x) sm.aux[i] = __ldg(q.aux + i);
  if (warp < q.n_bitmaps) {
    const ColDesc* cd = nullptr;
    for (int c = 0; c < q.n_cols; ++c)
      if (q.cols[c].bslot == warp) cd = &q.cols[c];
    const long long s0 = (long long)(t_begin * T);
    const unsigned long long cur = warp_count_below(cd->ends, cd->e64, cd->n, s0, cd->enc == ENC_INDEX);
    if (lane == 0) sm.tcur[warp] = cur;
  }
  __syncthreads();

  TileView tv;
  tv.bm = sm.bm;
  tv.pre = sm.pre;
  tv.cur = sm.tcur;
  tv.win = nullptr;
  tv.pbm = nullptr;
  tv.wn = sm.wcnt;   // zero: no windows in segment mode
  tv.stage = nullptr;
  tv.aux = aux_smem ? sm.aux : q.aux;
  tv.nwords = nwords;
  uint32_t rows_since_flush = 0;
  uint16_t* mylist = sm.clist + (warp < kWarps ? warp : 0) * (GPW * 32);
  const uint32_t wbase = warp * 32, gstride = kWarps * 32;

  unsigned long long* nextb = reinterpret_cast<unsigned long long*>(sm.win);
  const unsigned long long end_row = t_end * T < q.n_rows ? t_end * T : q.n_rows;
  for (unsigned long long t = t_begin; t < t_end; ++t) {
    const unsigned long long s = t * T;
    // ---- long segments: when no column has a boundary before the end of
    // this tile, the rows up to the first boundary of any column form one
    // aligned segment.  It is aggregated once and its tiles are skipped, so
    // the walk costs follow the runs rather than the rows (at most one flush
    // period per span, so the shared accumulators keep their bounds).
    if (threadIdx.x < q.n_bitmaps) {
      const int j = threadIdx.x;
      const ColDesc& cd = bitmap_col(q, j);
      const unsigned long long cur = sm.tcur[j];
      nextb[j] = cur < cd.n ? (unsigned long long)ldg_val(cd.ends, cur, cd.e64) : ~0ull;
    }
    __syncthreads();
    {
      unsigned long long m = ~0ull;
      for (int j = 0; j < q.n_bitmaps; ++j) m = nextb[j] < m ? nextb[j] : m;
      unsigned long long span_end = m < end_row ? m : end_row;
      const unsigned long long cap = s + (q.flush_rows - rows_since_flush);
      if (span_end > cap) span_end = cap;
      if (span_end >= s + T || (span_end == end_row && span_end > s)) {
        if (span_end != end_row) span_end = span_end / T * T;
        const unsigned long long L = span_end - s;
        if (threadIdx.x == 0) seg_span_update(q, sm, tv.aux, s, L);
        __syncthreads();
        if (threadIdx.x < q.n_bitmaps) {
          const int j = threadIdx.x;
          if (bitmap_col(q, j).enc == ENC_RLE && nextb[j] == span_end) sm.tcur[j] += 1;   // that run ended here
        }
        rows_since_flush += (uint32_t)L;
        t = (span_end + T - 1) / T - 1;   // the loop moves on to the tile holding span_end
        const bool need = (t + 1 == t_end) || (!q.table_dense && sm.misc[0] * 2 > (int)q.table_slots) ||
                          rows_since_flush + T > q.flush_rows;
        __syncthreads();
        if (need) {
          flush_table(q, sm);
          __syncthreads();
          if (threadIdx.x == 0) sm.misc[0] = 0;
          rows_since_flush = 0;
        }
        continue;
      }
    }
    const unsigned long long e = (s + T < q.n_rows) ? s + T : q.n_rows;
    const uint32_t rows = (uint32_t)(e - s);
    build_bitmaps(q, sm, s, e, nwords);
    build_segments(q, sm, nwords, rows);
    if (warp < kWarps) {
      const uint32_t pm = phase_filter<true, GPW>(q, tv, sm.seg, wbase, gstride, (uint32_t)sm.misc[2]);
      const uint32_t n_pass = compact<GPW>(pm, wbase, gstride, mylist);
      phase_aggregate<true, 2>(q, sm, tv, sm.seg, mylist, n_pass, s);
    }
    __syncthreads();
    if (threadIdx.x < q.n_bitmaps) {
      const int j = threadIdx.x;
      const uint32_t* P = sm.pre + j * (nwords + 1);
      sm.tcur[j] += P[nwords] + (unsigned long long)sm.flags[kMaxBitmapCols + j];
      sm.flags[j] = 0;
      sm.flags[kMaxBitmapCols + j] = 0;
    }
    rows_since_flush += rows;
    const bool need = (t + 1 == t_end) || (!q.table_dense && sm.misc[0] * 2 > (int)q.table_slots) ||
                      rows_since_flush + T > q.flush_rows;
    if (need) {
      flush_table(q, sm);
      __syncthreads();
      if (threadIdx.x == 0) sm.misc[0] = 0;
      rows_since_flush = 0;
    }
  }
}

}  // namespace cq

namespace cq {

// ------------------------------------------------------------------ walk by runs
// First index of sorted a[0, n) whose entry exceeds key (upper) or is at
// least key (lower); a plain binary search by one thread.
__device__ __forceinline__ unsigned long long thread_bound(const void* a, bool e64, unsigned long long n, long long key,
                                                          bool upper) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    const long long x = ldg_val(a, mid, e64);
    if (upper ? x <= key : x < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Segment mode without tiles (Section 6 alignment as a k-way merge of the
// columns' boundaries): thread u of the grid takes the u-th equal share of
// the entries (runs / listed rows) of the column with the most of them, i.e.
// the rows from its share's first entry to the next share's, clipped to the
// launch's rows [r_lo, r_hi).  It finds every column's run / next listed row
// at its first row by binary search, then walks its rows segment by segment:
// the segment ends at the nearest boundary of any column (a listed row is a
// segment of its own), is aggregated once (segment_update) and the columns
// whose boundary it reached advance.  The work follows the runs, not the
// rows.  Per-thread cursors live in shared memory (dynamic column index).
__device__ inline void run_range(const QueryDesc& q, const Smem& sm, const uint32_t* aux, unsigned long long r_lo,
                                 unsigned long long r_hi) {
  const int nb = q.n_bitmaps;
  const unsigned long long U = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const ColDesc& D = bitmap_col(q, q.run_slot);
  const unsigned long long nD = D.n;
  unsigned long long r0, r1;
  if (nD == 0) {   // no entries anywhere: one thread takes every row
    r0 = u == 0 ? 0ull : q.n_rows;
    r1 = q.n_rows;
  } else {
    const unsigned long long a = u * nD / U, b = (u + 1) * nD / U;
    auto start_row = [&](unsigned long long i) -> unsigned long long {
      if (i == 0) return 0ull;
      if (i >= nD) return q.n_rows;
      return D.enc == ENC_RLE ? (unsigned long long)ldg_val(D.ends, i - 1, D.e64)
                              : (unsigned long long)ldg_val(D.ends, i, D.e64);
    };
    r0 = start_row(a);
    r1 = start_row(b);
  }
  if (r0 < r_lo) r0 = r_lo;
  if (r1 > r_hi) r1 = r_hi;
  if (r0 >= r1) return;
  // per column j: cursor, next boundary (RLE: end of the current run; index:
  // next listed row, ~0 past the last), value (RLE: run value; index: listed)
  unsigned long long* cur = reinterpret_cast<unsigned long long*>(sm.win) + threadIdx.x;
  long long* bnd = reinterpret_cast<long long*>(sm.win) + (size_t)nb * blockDim.x + threadIdx.x;
  long long* val = reinterpret_cast<long long*>(sm.win) + (size_t)2 * nb * blockDim.x + threadIdx.x;
  const size_t S = blockDim.x;
  auto load = [&](int j) {
    const ColDesc& c = bitmap_col(q, j);
    const unsigned long long k = cur[j * S];
    if (k < c.n) {
      bnd[j * S] = ldg_val(c.ends, k, c.e64);
      val[j * S] = ldg_val(c.vals, k, c.v64);
    } else {
      bnd[j * S] = c.enc == ENC_RLE ? (long long)q.n_rows : LLONG_MAX;
      val[j * S] = 0;
    }
  };
  for (int j = 0; j < nb; ++j) {
    const ColDesc& c = bitmap_col(q, j);
    cur[j * S] = thread_bound(c.ends, c.e64, c.n, (long long)r0, c.enc == ENC_RLE);
    load(j);
  }
  unsigned long long pos = r0;
  while (pos < r1) {
    unsigned long long nxt = r1;
    for (int j = 0; j < nb; ++j) {
      const unsigned long long x = (unsigned long long)bnd[j * S];
      if (bitmap_col(q, j).enc == ENC_INDEX && x == pos) nxt = pos + 1 < nxt ? pos + 1 : nxt;
      else if (x < nxt) nxt = x;
    }
    auto value = [&](int c) -> long long {
      const ColDesc& cd = q.cols[c];
      const int j = cd.bslot;
      if (cd.enc == ENC_RLE) return val[j * S];
      return (unsigned long long)bnd[j * S] == pos ? val[j * S] : cd.base;
    };
    auto listed = [&](int c, long long* v) {
      const int j = q.cols[c].bslot;
      if ((unsigned long long)bnd[j * S] != pos) return false;
      *v = val[j * S];
      return true;
    };
    segment_update(q, sm, aux, pos, nxt - pos, value, listed);
    for (int j = 0; j < nb; ++j) {
      const ColDesc& c = bitmap_col(q, j);
      const unsigned long long x = (unsigned long long)bnd[j * S];
      if ((c.enc == ENC_RLE && x == nxt) || (c.enc == ENC_INDEX && x == pos)) {
        cur[j * S] += 1;
        load(j);
      }
    }
    pos = nxt;
  }
}

}  // namespace cq
