// cq_rowpath.cuh -- row-mode steps of the fused query: the helper warp's
// bitmap builder with its prefetch windows, and the pipelined walk over a
// range of tiles.  Used by the one-query kernel (cq_row.cu) and by the
// persistent batch kernel (cq_batch.cu).
#pragma once

#include "cq_phases.cuh"

namespace cq {

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// helper-warp state lives in the (otherwise unused) flags / misc words:
// hcur[j] = first run / position of bitmap column j in the next tile to build
__device__ __forceinline__ unsigned long long* helper_cursor(const Smem& sm) {
  return reinterpret_cast<unsigned long long*>(sm.flags);
}

// Window set `wb`: per bitmap column kWin run ends / positions, then the
// values of the same runs / listed rows.
__device__ __forceinline__ uint8_t* window_set(const QueryDesc& q, const Smem& sm, int wb) {
  return sm.win + (size_t)wb * q.n_bitmaps * kWin * 16;
}
__device__ __forceinline__ uint8_t* window(const QueryDesc& q, const Smem& sm, int wb, int j) {
  return window_set(q, sm, wb) + (size_t)j * kWin * 16;
}

// Prefetch kWin run ends / positions and their values of every bitmap
// column, from the helper cursor on, into window set `wb` (helper warp).
__device__ inline void prefetch_windows(const QueryDesc& q, const Smem& sm, int wb) {
  const int lane = threadIdx.x & 31;
  const unsigned long long* hcur = helper_cursor(sm);
  for (int j = 0; j < q.n_bitmaps; ++j) {
    const ColDesc& cd = bitmap_col(q, j);
    const unsigned long long cur = hcur[j];
    const uint32_t avail = cur < cd.n ? (uint32_t)((cd.n - cur) < kWin ? (cd.n - cur) : kWin) : 0u;
    uint8_t* dst = window(q, sm, wb, j);
    uint8_t* vdst = dst + kWin * 8;
    for (uint32_t i = lane; i < avail; i += 32) {
      if (cd.e64) cp_async8(dst + 8 * i, reinterpret_cast<const long long*>(cd.ends) + cur + i);
      else cp_async4(dst + 4 * i, reinterpret_cast<const int*>(cd.ends) + cur + i);
      if (cd.v64) cp_async8(vdst + 8 * i, reinterpret_cast<const long long*>(cd.vals) + cur + i);
      else cp_async4(vdst + 4 * i, reinterpret_cast<const int*>(cd.vals) + cur + i);
    }
    if (lane == 0) sm.wcnt[wb * kMaxBitmapCols + j] = avail;
  }
  cp_async_commit();
}

// Build the bitmaps of tile [s, e) into buffer `buf` from the prefetched
// windows (falling back to global loads past a window), record the tile's
// start cursors and advance the helper cursors (helper warp).
__device__ inline void helper_build(const QueryDesc& q, const Smem& sm, int buf, int wb, unsigned long long s,
                                    unsigned long long e, uint32_t nwords) {
  const int lane = threadIdx.x & 31;
  const int nb = q.n_bitmaps;
  unsigned long long* hcur = helper_cursor(sm);
  cp_async_wait_all();
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    const ColDesc& cd = bitmap_col(q, j);
    const bool is_rle = cd.enc == ENC_RLE;
    uint32_t* B = sm.bm + ((size_t)buf * nb + j) * nwords;
    uint32_t* P = sm.pre + ((size_t)buf * nb + j) * (nwords + 1);
    for (uint32_t w = lane; w < nwords; w += 32) B[w] = 0;
    __syncwarp();
    const unsigned long long cur = hcur[j];
    const uint32_t avail = cur < cd.n ? (uint32_t)((cd.n - cur) < kWin ? (cd.n - cur) : kWin) : 0u;
    const uint8_t* win = window(q, sm, wb, j);
    unsigned long long cnt = 0;
    int eq = 0;
    for (unsigned long long base = 0;; base += 32) {
      const unsigned long long idx = cur + base + lane;
      long long x = 0;
      bool have = true;
      if (base + lane < avail) {
        x = cd.e64 ? reinterpret_cast<const long long*>(win)[base + lane]
                   : (long long)reinterpret_cast<const int*>(win)[base + lane];
      } else if (idx < cd.n) {
        x = ldg_val(cd.ends, idx, cd.e64);
      } else {
        have = false;
      }
      const bool in_tile = have && (unsigned long long)x < e;
      if (in_tile) {
        // a boundary before the tile would mean a corrupt cursor: flag it, never write
        if ((unsigned long long)x < s || (is_rle && (unsigned long long)x == s)) {
          report(q, CQ_ERR_INVALID_ARG, 2ull + ((unsigned long long)j << 8), s, (unsigned long long)x);
        } else {
          const uint32_t o = (uint32_t)((unsigned long long)x - s);
          atomicOr(&B[o >> 5], 1u << (o & 31));
        }
      }
      const uint32_t stop = __ballot_sync(0xFFFFFFFFu, !in_tile);
      if (stop) {
        const int f = __ffs(stop) - 1;
        cnt = base + f;
        const long long xf = __shfl_sync(0xFFFFFFFFu, x, f);
        const bool hf = __shfl_sync(0xFFFFFFFFu, have, f);
        eq = (is_rle && hf && (unsigned long long)xf == e) ? 1 : 0;
        break;
      }
    }
    __syncwarp();
    // word prefix popcounts
    const uint32_t per = nwords / 32;
    uint32_t local = 0;
    for (uint32_t k = 0; k < per; ++k) local += __popc(B[lane * per + k]);
    uint32_t incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t run = incl - local;
    for (uint32_t k = 0; k < per; ++k) {
      P[lane * per + k] = run;
      run += __popc(B[lane * per + k]);
    }
    if (lane == 31) P[nwords] = incl;
    if (lane == 0) {
      sm.tcur[buf * kMaxBitmapCols + j] = cur;
      hcur[j] = cur + cnt + (unsigned long long)eq;
    }
    __syncwarp();
  }
}

// NCW compute warps (+1 helper); GPW groups of 32 rows per compute warp, so a
// tile holds NCW * GPW * 32 rows.  MINB CTAs share an SM (registers are
// capped so that MINB CTAs fit).

// Set bits [a, b) of a tile bitmap (this lane's run; its interior words are
// its own, its end words may be shared with neighbouring runs).
__device__ __forceinline__ void fill_bits(uint32_t* B, uint32_t a, uint32_t b) {
  if (a >= b) return;
  const uint32_t wa = a >> 5, wz = (b - 1) >> 5;
  const uint32_t ma = ~0u << (a & 31), mz = ~0u >> (31 - ((b - 1) & 31));
  if (wa == wz) {
    atomicOr(&B[wa], ma & mz);
    return;
  }
  atomicOr(&B[wa], ma);
  for (uint32_t w = wa + 1; w < wz; ++w) B[w] = ~0u;
  atomicOr(&B[wz], mz);
}

// Fill the pass bitmaps of tile [s, e) in buffer `buf` from the window set
// `wb` (helper warp, after helper_build of the same tile): each predicate on
// an RLE column is evaluated once per run of the tile and sets the run's
// rows; one on an index column is evaluated once for the default and once
// per listed row.
__device__ inline void helper_pass_bitmaps(const QueryDesc& q, const Smem& sm, const uint32_t* aux, int buf, int wb,
                                           unsigned long long s, unsigned long long e, uint32_t nwords) {
  const int lane = threadIdx.x & 31;
  const uint32_t rows = (uint32_t)(e - s);
  const int nb = q.n_bitmaps;
  for (int pi = 0; pi < q.n_preds; ++pi) {
    const PredDesc& p = q.preds[pi];
    if (p.pbm == 0xFF) continue;
    const ColDesc& c = q.cols[p.col];
    const int j = c.bslot;
    uint32_t* PB = sm.pbm + ((size_t)buf * q.n_pbm + p.pbm) * nwords;
    const uint32_t nset = sm.pre[((size_t)buf * nb + j) * (nwords + 1) + nwords];
    const unsigned long long cur = sm.tcur[buf * kMaxBitmapCols + j];
    const uint8_t* win = window(q, sm, wb, j);
    const uint32_t avail = sm.wcnt[wb * kMaxBitmapCols + j];
    auto end_at = [&](uint32_t k) -> unsigned long long {
      if (k < avail) return c.e64 ? (unsigned long long)reinterpret_cast<const long long*>(win)[k]
                                  : (unsigned long long)reinterpret_cast<const int*>(win)[k];
      return (unsigned long long)ldg_val(c.ends, cur + k, c.e64);
    };
    auto val_at = [&](uint32_t k) -> long long {
      if (k < avail) {
        const uint8_t* v = win + kWin * 8;
        return c.v64 ? reinterpret_cast<const long long*>(v)[k] : (long long)reinterpret_cast<const int*>(v)[k];
      }
      return ldg_val(c.vals, cur + k, c.v64);
    };
    if (c.enc == ENC_RLE) {
      for (uint32_t w = lane; w < nwords; w += 32) PB[w] = 0u;
      __syncwarp();
      // nset boundaries inside the tile: nset + 1 runs, the last one clipped
      for (uint32_t k = lane; k <= nset; k += 32) {
        const uint32_t a = k == 0 ? 0u : (uint32_t)(end_at(k - 1) - s);
        const unsigned long long x = end_at(k);
        const uint32_t b = x - s < rows ? (uint32_t)(x - s) : rows;
        if (pred_eval(p, aux, val_at(k))) fill_bits(PB, a, b);
      }
    } else {
      const bool base_pass = pred_eval(p, aux, c.base);
      for (uint32_t w = lane; w < nwords; w += 32) {
        const uint32_t lo = w * 32;
        uint32_t m = base_pass ? ~0u : 0u;
        if (lo >= rows) m = 0u;
        else if (rows - lo < 32) m &= (1u << (rows - lo)) - 1u;
        PB[w] = m;
      }
      __syncwarp();
      for (uint32_t k = lane; k < nset; k += 32) {
        const uint32_t o = (uint32_t)(end_at(k) - s);
        if (pred_eval(p, aux, val_at(k)) != base_pass) atomicXor(&PB[o >> 5], 1u << (o & 31));
      }
    }
    __syncwarp();
  }
}

// Walk tiles [t_begin, t_end) of one row-mode query with NCW compute warps
// and one helper warp (warp NCW): reset the group table, start the bulk-copy
// pipeline, then per tile filter and aggregate (compute warps) while the
// helper builds the next tile's bitmaps; flush the table when it fills and
// after the last tile.  Every issued stage is consumed before returning.
// The compute warps' work on one tile -- filter its rows, compact the passing
// ones, aggregate them -- is Body::tile; GenericBody reads every shape
// property of the query from its descriptor at run time (FastBody in
// cq_fast.cuh has them as compile-time constants).
// The helper warp's steps go through the body too: issue (lane 0: the bulk
// copies of tile u into stage st), prefetch (windows of run ends / positions
// into window set wb) and build (bitmaps and pass bitmaps of tile [s, e)).
struct GenericBody {
  template <int NCW, int GPW>
  __device__ static __forceinline__ void tile(const QueryDesc& q, const Smem& sm, const TileView& tv, uint32_t wbase,
                                              uint32_t rows, uint16_t* list, unsigned long long row0) {
    const uint32_t gstride = NCW * 32;
    const uint32_t pm = phase_filter<false, GPW>(q, tv, nullptr, wbase, gstride, rows);
    const uint32_t n_pass = compact<GPW>(pm, wbase, gstride, list);
    phase_aggregate<false, 2>(q, sm, tv, nullptr, list, n_pass, row0);
  }

  __device__ static __forceinline__ void issue(const QueryDesc& q, const Smem& sm, unsigned long long u, uint32_t st) {
    const uint32_t T = q.tile_rows;
    uint8_t* dst = sm.stage + (size_t)st * q.stage_bytes;
    const unsigned long long r0 = u * T;
    const unsigned long long rows = (q.n_rows - r0) < (unsigned long long)T ? (q.n_rows - r0) : (unsigned long long)T;
    uint32_t total = 0;
    for (int i = 0; i < q.n_row_cols; ++i) {
      const ColDesc& c = q.cols[q.row_cols[i]];
      const uint32_t bits = c.enc == ENC_PLAIN ? (c.v64 ? 64u : 32u) : (uint32_t)c.bw;
      total += (uint32_t)(((rows * bits + 7) / 8 + 15) / 16 * 16);
    }
    mbar_arrive_expect_tx(&sm.mbar[st], total);
    for (int i = 0; i < q.n_row_cols; ++i) {
      const ColDesc& c = q.cols[q.row_cols[i]];
      const uint32_t bits = c.enc == ENC_PLAIN ? (c.v64 ? 64u : 32u) : (uint32_t)c.bw;
      const uint32_t bytes = (uint32_t)(((rows * bits + 7) / 8 + 15) / 16 * 16);
      bulk_g2s(dst + c.stage_off, reinterpret_cast<const uint8_t*>(c.vals) + r0 * bits / 8, bytes, &sm.mbar[st]);
    }
  }

  // (one helper warp: hw = 0, nh = 1)
  __device__ static __forceinline__ void prefetch(const QueryDesc& q, const Smem& sm, int wb, int hw, int nh) {
    prefetch_windows(q, sm, wb);
  }

  __device__ static __forceinline__ void build(const QueryDesc& q, const Smem& sm, const uint32_t* aux, int buf, int wb,
                                               unsigned long long s, unsigned long long e, int hw, int nh) {
    const uint32_t nwords = q.tile_rows / 32;
    helper_build(q, sm, buf, wb, s, e, nwords);
    if (q.n_pbm) helper_pass_bitmaps(q, sm, aux, buf, wb, s, e, nwords);
  }
};

// NH helper warps (warps NCW .. NCW + NH - 1) share the bitmap columns:
// helper hw builds and prefetches columns j with j % NH == hw; helper 0 also
// issues the bulk copies.
template <int NCW, int GPW, class Body = GenericBody, int NH = 1>
__device__ __forceinline__ void row_range(const QueryDesc& q, const Smem& sm, unsigned long long t_begin,
                                          unsigned long long t_end) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t T = q.tile_rows;
  const uint32_t nwords = T / 32;
  const bool helper = warp >= NCW;
  const int hw = warp - NCW;
  const int nb = q.n_bitmaps;

  // ---- init: group table, aux tables, barriers, helper cursors
  for (uint32_t sl = threadIdx.x; sl < q.table_slots; sl += blockDim.x) reset_slot(q, sm, sl);
  if (threadIdx.x < 8) sm.misc[threadIdx.x] = 0;
  const bool aux_smem = q.aux_words <= kAuxSmemWords;
  if (aux_smem)
    for (uint32_t i = threadIdx.x; i < q.aux_words; i += blockDim.x) sm.aux[i] = __ldg(q.aux + i);
  if (threadIdx.x == 0) {
    for (int st = 0; st < q.stages; ++st) mbar_init(&sm.mbar[st], 1);
    fence_barrier_init();
  }
  if (helper) {
    for (int j = hw; j < nb; j += NH) {
      const ColDesc& cd = bitmap_col(q, j);
      // RLE: first run whose exclusive end exceeds the first row; index: first position >= it
      const unsigned long long c0 =
          warp_count_below(cd.ends, cd.e64, cd.n, (long long)(t_begin * T), cd.enc == ENC_INDEX);
      if (lane == 0) helper_cursor(sm)[j] = c0;
    }
  }
  __syncthreads();

  // ---- bulk-copy producer (helper lane 0): stage st holds tile u; stage and
  // barrier parity advance with the tile (no division per tile)
  // ---- prologue: first tile's bitmaps, windows of the second, the first stages
  if (helper) {
    if (hw == 0 && lane == 0)
      for (unsigned long long u = t_begin; u < t_end && u < t_begin + q.stages; ++u)
        Body::issue(q, sm, u, (uint32_t)(u - t_begin));
    if (nb) {
      // window set (u - t_begin) % kWinBufs serves tile u: prefetched two
      // tiles ahead, turned into bitmaps one tile ahead, read by the compute
      // warps (values) while the tile is processed
      Body::prefetch(q, sm, 0, hw, NH);
      const unsigned long long e0 = ((t_begin + 1) * T < q.n_rows) ? (t_begin + 1) * T : q.n_rows;
      Body::build(q, sm, aux_smem ? sm.aux : q.aux, 0, 0, t_begin * T, e0, hw, NH);
      if (t_begin + 1 < t_end) Body::prefetch(q, sm, 1, hw, NH);
    }
  }
  __syncthreads();

  uint32_t rows_since_flush = 0;
  // line mode: the first run ordinal of key 0's column whose line has not
  // been flushed (every thread tracks it).  While tile t is aggregated, the
  // compute warps flush the lines of the runs that ended before it,
  // [line_base, first run of t), so after its barrier line_base is tile t's
  // first run; a full flush moves it to the next tile's first run.
  unsigned long long line_base = q.line_mode ? sm.tcur[q.line_slot] : 0ull;
  uint16_t* mylist = sm.clist + (helper ? 0 : warp) * (GPW * 32);
  const uint32_t wbase = warp * 32;
  uint32_t st = 0, ph = 0;   // stage of tile t and the parity of its barrier phase
  uint32_t wbi = 0;          // window set of tile t: (t - t_begin) % kWinBufs

  for (unsigned long long t = t_begin; t < t_end; ++t) {
    const unsigned long long s = t * T;
    const unsigned long long e = (s + T < q.n_rows) ? s + T : q.n_rows;
    const uint32_t rows = (uint32_t)(e - s);
    const int buf = (int)((t - t_begin) & 1ull);
    if (!helper) {
      mbar_wait_bounded(&sm.mbar[st], ph, q.err);
      TileView tv;
      tv.bm = sm.bm + (size_t)buf * nb * nwords;
      tv.pre = sm.pre + (size_t)buf * nb * (nwords + 1);
      tv.cur = sm.tcur + buf * kMaxBitmapCols;
      const int wb = (int)wbi;
      tv.win = window_set(q, sm, wb);
      tv.pbm = sm.pbm + (size_t)buf * q.n_pbm * nwords;
      tv.wn = sm.wcnt + wb * kMaxBitmapCols;
      tv.stage = sm.stage + (size_t)st * q.stage_bytes;
      tv.aux = aux_smem ? sm.aux : q.aux;
      tv.nwords = nwords;
      tv.line_base = line_base;
      Body::template tile<NCW, GPW>(q, sm, tv, wbase, rows, mylist, s);
    } else if (nb && t + 1 < t_end) {
      const int wb1 = (int)(wbi + 1 == kWinBufs ? 0 : wbi + 1);
      const unsigned long long e1 = (e + T < q.n_rows) ? e + T : q.n_rows;
      Body::build(q, sm, aux_smem ? sm.aux : q.aux, buf ^ 1, wb1, e, e1, hw, NH);
      if (t + 2 < t_end) Body::prefetch(q, sm, (int)(wbi == 0 ? 2 : wbi - 1), hw, NH);
    }
    // one barrier per tile; thread 0 decides the flush from the occupancy it
    // sees (an early or late flush is harmless: a full table falls back to
    // the global accumulators)
    rows_since_flush += rows;
    const bool last = t + 1 == t_end;
    // line mode: the helper that built tile t + 1's bitmaps of key 0's column
    // asks for a full flush when that tile's last run would share a line with
    // a run not flushed by then (tile t's first run or later: ordinal
    // difference >= lines)
    bool lines_full = false;
    // tile t's first run: read before the barrier (the helper rebuilds this
    // buffer for tile t + 2 once past it)
    const unsigned long long first_run_t = q.line_mode ? sm.tcur[buf * kMaxBitmapCols + q.line_slot] : 0ull;
    if (q.line_mode && helper && lane == 0 && hw == (int)q.line_slot % NH && !last) {
      const int b1 = buf ^ 1;
      const unsigned long long last_ord =
          sm.tcur[b1 * kMaxBitmapCols + q.line_slot] + sm.pre[((size_t)b1 * nb + q.line_slot) * (nwords + 1) + nwords];
      lines_full = last_ord - first_run_t >= (1ull << q.line_log2);
    }
    const int need = __syncthreads_or(lines_full ||
                                      (threadIdx.x == 0 &&
                                       (last || (!q.table_dense && !q.line_mode && sm.misc[0] * 2 > (int)q.table_slots) ||
                                        rows_since_flush + T > q.flush_rows)));
    // tile t's stage is free: refill it with tile t + stages
    if (helper && hw == 0 && lane == 0 && t + q.stages < t_end) Body::issue(q, sm, t + q.stages, st);
    if (q.line_mode) line_base = first_run_t;
    if (need) {
      flush_table(q, sm);
      if (threadIdx.x == 0) sm.misc[0] = 0;
      __syncthreads();
      rows_since_flush = 0;
      if (q.line_mode && !last) line_base = sm.tcur[(buf ^ 1) * kMaxBitmapCols + q.line_slot];
    }
    if (++st == q.stages) {
      st = 0;
      ph ^= 1u;
    }
    wbi = wbi + 1 == kWinBufs ? 0 : wbi + 1;
  }
  // the stage barriers are dead: invalidate them so the batch kernel may
  // reuse their words for another query's layout
  if (threadIdx.x == 0)
    for (int st = 0; st < q.stages; ++st) mbar_inval(&sm.mbar[st]);
}

}  // namespace cq
