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

// One aligned segment of L rows starting at row s over which every column is
// constant: each RLE column holds the run at its cursor, each index column its
// default (no listed row inside).  Filter and aggregate it once: COUNT += L,
// SUM += value x L, MIN / MAX on the value (Section 7; the rows need no
// bitmaps).  One thread.
__device__ inline void seg_span_update(const QueryDesc& q, const Smem& sm, const uint32_t* aux, unsigned long long s,
                                       unsigned long long L) {
  auto value = [&](const ColDesc& c) -> long long {
    if (c.enc == ENC_RLE) return ldg_val(c.vals, sm.tcur[c.bslot], c.v64);
    return c.base;   // index column, unlisted rows
  };
  for (int i = 0; i < q.n_preds; ++i)
    if (!pred_eval(q.preds[i], aux, value(q.cols[q.preds[i].col]))) return;
  unsigned long long gid = 0;
  for (int ki = 0; ki < q.n_keys; ++ki) {
    const KeyDesc& k = q.keys[ki];
    const long long v = value(q.cols[k.col]);
    unsigned long long d;
    if (!key_digit(k, aux, v, &d)) {
      report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)ki << 8), s, (unsigned long long)v);
      return;
    }
    gid += d * k.stride;
  }
  int slot = q.n_groups == 1 && !q.ghash ? 0 : table_slot(q, sm, gid);
  uint32_t gi = 0;
  if (slot >= 0) {
    atomicAdd(scount(q, sm, slot), (unsigned)L);
  } else {
    const long long g = gindex(q, gid);
    if (g < 0) return;
    gi = (uint32_t)g;
    atomicAdd(gword(q, 0, gi), L);
  }
  for (int ai = 0; ai < q.n_aggs; ++ai) {
    const AggDesc& a = q.aggs[ai];
    // index-column aggregates see no listed row here; finalize adds the
    // default from COUNT
    if (a.kind == AK_SUM) sum_add(q, sm, a, slot, gi, mul_s64(value(q.cols[a.col]), (long long)L));
    else if (a.kind == AK_MIN || a.kind == AK_MAX) minmax_add(q, sm, a, slot, gi, value(q.cols[a.col]), a.kind == AK_MIN);
  }
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
