// cq_fast.cuh -- the compute warps' tile body of the row-mode kernel with the
// query's shape known at compile time.
//
// The generic body (GenericBody in cq_rowpath.cuh) interprets the query
// descriptor: which encoding each column has, which test each predicate
// makes, how keys and aggregates are laid out.  Here every such property is a
// compile-time constant of the shape class S (generated per query shape and
// compiled at run time, cq_jit.cu), so the filter and the aggregation become
// straight-line code: no descriptor dispatch, constant bit widths and
// stage offsets, one shared-memory read per packed field.  Literal values
// (range bounds, IN tables, key minima and strides, bases) stay in the
// descriptor, so queries that differ only in their literals share a kernel.
//
// The helper warp's steps (bulk-copy issue, window prefetch, bitmap and
// pass-bitmap building) are specialised the same way.
//
// S provides (all constexpr): tile_rows, n_cols, n_bitmaps, n_row_cols,
// stage_bytes, n_preds, n_pbm, n_keys, n_aggs, one_group, table_dense, ghash
// (groups in the global hash table, 64-bit packed keys), line_mode (the
// shared table holds one line per run of key 0's RLE column); per
// column c: enc, v64, e64, bw, bslot, raw_off, stage_off; bcol(j), the
// column of bitmap slot j; row_col(i), the i-th staged column; per predicate
// i (evaluation order): pcol, pkind, pn32, ppbm, pneg (complemented), pcl
// (PC_ALONE / PC_MEMBER / PC_LAST: its place in its clause);
// per key k: kcol, kremap, kn32; per aggregate i: akind, acol, asw, awide,
// asw32, agw, ared32, aw32, an32, as32, asrc (the first aggregate reading the
// same column value, whose read is reused), aub (SUM inputs in [0, 2^aub)).
#pragma once

#include "cq_rowpath.cuh"

namespace cq {

template <bool B, class T, class F>
struct Pick {
  typedef T type;
};
template <class T, class F>
struct Pick<false, T, F> {
  typedef F type;
};

template <int I, int N, class F>
__device__ __forceinline__ void static_for_from(F& f) {
  if constexpr (I < N) {
    f(IC<I>());
    static_for_from<I + 1, N>(f);
  }
}

// f(IC<0>()), ..., f(IC<N-1>()): a loop whose index is a constant expression.
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_from<0, N>(f);
}

// Field o of an LSB-first bit stream of BW-bit fields (shared memory).
template <int BW>
__device__ __forceinline__ uint64_t field_of(const uint32_t* w, uint32_t o) {
  const uint32_t bit = o * (uint32_t)BW;
  const uint32_t q = bit >> 5, sh = bit & 31;
  const uint32_t lo = __funnelshift_r(w[q], w[q + 1], sh);
  if constexpr (BW == 32) {
    return lo;
  } else if constexpr (BW < 32) {
    return lo & ((1u << BW) - 1u);
  } else {
    const uint32_t hi = __funnelshift_r(w[q + 1], w[q + 2], sh);
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    if constexpr (BW == 64) return v;
    else return v & ((1ull << BW) - 1ull);
  }
}

// Raw value (see col_raw) of column C at tile row o.
template <class S, int C>
__device__ __forceinline__ long long fast_raw(const QueryDesc& q, const TileView& t, uint32_t o) {
  constexpr int E = S::enc(C);
  if constexpr (E == ENC_PLAIN) {
    const uint8_t* p = t.stage + S::stage_off(C);
    if constexpr (S::v64(C)) return reinterpret_cast<const long long*>(p)[o];
    else return (long long)reinterpret_cast<const int*>(p)[o];
  } else if constexpr (E == ENC_PACKED || E == ENC_DICT) {
    const uint64_t f = field_of<S::bw(C)>(reinterpret_cast<const uint32_t*>(t.stage + S::stage_off(C)), o);
    if constexpr (S::raw_off(C)) return (long long)f;
    else return (long long)(f + (uint64_t)q.cols[C].base);
  } else {
    return col_raw<E>(q.cols[C], t, o);
  }
}

// 32-bit raw value; only for columns the planner marked narrow.
template <class S, int C>
__device__ __forceinline__ int fast_raw32(const QueryDesc& q, const TileView& t, uint32_t o) {
  constexpr int E = S::enc(C);
  if constexpr (E == ENC_PLAIN) {
    return reinterpret_cast<const int*>(t.stage + S::stage_off(C))[o];
  } else if constexpr (E == ENC_PACKED || E == ENC_DICT) {
    return (int)(uint32_t)field_of<S::bw(C)>(reinterpret_cast<const uint32_t*>(t.stage + S::stage_off(C)), o);
  } else {
    return col_raw32<E>(q.cols[C], t, o);
  }
}

// Reader of one staged row-level column for this lane's rows of a tile:
// group g holds row wbase + g * GS + lane.  The lane's first bit (element)
// is computed once; every later group is a constant word offset from it.
template <class S, int C, uint32_t GS>
struct GroupReader {
  const uint8_t* p;
  uint32_t b0;
  __device__ __forceinline__ GroupReader(const TileView& t, uint32_t wbase) {
    p = t.stage + S::stage_off(C);
    const uint32_t o = wbase + (threadIdx.x & 31);
    if constexpr (S::enc(C) == ENC_PLAIN) b0 = o;
    else b0 = o * (uint32_t)S::bw(C);
  }
  __device__ __forceinline__ int raw32(int g) const {
    if constexpr (S::enc(C) == ENC_PLAIN) {
      return reinterpret_cast<const int*>(p)[b0 + g * GS];
    } else {
      constexpr uint32_t BW = S::bw(C);
      const uint32_t* w = reinterpret_cast<const uint32_t*>(p) + (b0 >> 5) + g * (GS / 32 * BW);
      const uint32_t lo = __funnelshift_r(w[0], w[1], b0 & 31);
      if constexpr (BW >= 32) return (int)lo;
      else return (int)(lo & ((1u << BW) - 1u));
    }
  }
  __device__ __forceinline__ long long raw64(const QueryDesc& q, int g) const {
    if constexpr (S::enc(C) == ENC_PLAIN) {
      if constexpr (S::v64(C)) return reinterpret_cast<const long long*>(p)[b0 + g * GS];
      else return (long long)reinterpret_cast<const int*>(p)[b0 + g * GS];
    } else {
      constexpr uint32_t BW = S::bw(C);
      const uint32_t* w = reinterpret_cast<const uint32_t*>(p) + (b0 >> 5) + g * (GS / 32 * BW);
      const uint32_t sh = b0 & 31;
      uint64_t f = __funnelshift_r(w[0], w[1], sh);
      if constexpr (BW > 32) f |= (uint64_t)__funnelshift_r(w[1], w[2], sh) << 32;
      if constexpr (BW < 64) f &= (BW == 64 ? ~0ull : ((1ull << BW) - 1ull));
      if constexpr (S::raw_off(C)) return (long long)f;
      else return (long long)(f + (uint64_t)q.cols[C].base);
    }
  }
};

// ------------------------------------------------------------------ filter
// Bit g of the result: row wbase + g * GS + lane passes the filter, the
// conjunction of clauses (Section 5: AND, OR, NOT).  A predicate alone in
// its clause ANDs its result into the mask directly; a clause's members OR
// theirs into `acc`, which the last member ANDs in.  A complemented
// predicate's test is inverted here; its pass bitmap already holds the
// complement.
template <class S, uint32_t GS, int GPW>
__device__ __forceinline__ uint32_t fast_filter(const QueryDesc& q, const TileView& t, uint32_t wbase, uint32_t rows) {
  const int lane = threadIdx.x & 31;
  uint32_t valid = 0;
#pragma unroll
  for (int g = 0; g < GPW; ++g) valid |= (wbase + g * GS + lane < rows ? 1u : 0u) << g;
  uint32_t pm = valid, acc = 0;
  static_for<S::n_preds>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int kind = S::pkind(i);
    constexpr int c = S::pcol(i);
    constexpr int E = S::enc(c);
    constexpr int cl = S::pcl(i);
    constexpr bool ng = S::pneg(i);
    // row group g's result for this predicate (`ok` before any complement)
    auto put = [&](int g, bool ok, bool complement) {
      if (complement) ok = !ok;
      if constexpr (cl == PC_ALONE) pm &= ok ? ~0u : ~(1u << g);
      else acc |= (ok ? 1u : 0u) << g;
    };
    if constexpr (S::ppbm(i) != 0xFF) {
      // evaluated once per run / listed row by the helper warp: one bit per row
      const uint32_t* PB = t.pbm + (size_t)S::ppbm(i) * (S::tile_rows / 32);
#pragma unroll
      for (int g = 0; g < GPW; ++g) put(g, (PB[(wbase + g * GS) >> 5] >> lane) & 1u, false);
    } else if constexpr (kind == PK_FALSE) {
      if constexpr (cl == PC_ALONE) pm = 0;
    } else if constexpr (kind == PK_TRUE) {
      if constexpr (cl != PC_ALONE) acc = ~0u;
    } else {
      if (!__any_sync(0xFFFFFFFFu, pm != 0)) return;
      const PredDesc& p = q.preds[i];
      if constexpr (E == ENC_RLE || E == ENC_INDEX) {
        // per-row lookups through the tile bitmaps (more run-column
        // predicates than pass bitmaps)
#pragma unroll 4
        for (int g = 0; g < GPW; ++g) {
          const uint32_t o = wbase + g * GS + lane;
          bool ok;
          if constexpr (S::pn32(i)) {
            if constexpr (kind == PK_RANGE) ok = pred_test32<PT_RANGE32>(p, t.aux, col_raw32<E>(q.cols[c], t, o));
            else if constexpr (kind == PK_NE) ok = pred_test32<PT_NE32>(p, t.aux, col_raw32<E>(q.cols[c], t, o));
            else ok = pred_test32<PT_BITMAP32>(p, t.aux, col_raw32<E>(q.cols[c], t, o));
          } else {
            const long long v = col_raw<E>(q.cols[c], t, o);
            if constexpr (kind == PK_RANGE) ok = pred_test<PT_RANGE>(p, t.aux, v);
            else if constexpr (kind == PK_NE) ok = pred_test<PT_NE>(p, t.aux, v);
            else if constexpr (kind == PK_BITMAP) ok = pred_test<PT_BITMAP>(p, t.aux, v);
            else ok = pred_test<PT_LIST>(p, t.aux, v);
          }
          put(g, ok, ng);
        }
      } else {
        const GroupReader<S, c, GS> rd(t, wbase);
        if constexpr (S::pn32(i)) {
          const uint32_t lo = (uint32_t)p.lo32, span = (uint32_t)p.hi32 - (uint32_t)p.lo32;
          const uint32_t* bm = t.aux + p.aux_off;
#pragma unroll
          for (int g = 0; g < GPW; ++g) {
            const uint32_t v = (uint32_t)rd.raw32(g);
            bool ok;
            if constexpr (kind == PK_RANGE) {
              ok = v - lo <= span;
            } else if constexpr (kind == PK_NE) {
              ok = v != lo;
            } else {  // PK_BITMAP
              const uint32_t d = v - lo;
              ok = d <= span && ((bm[d >> 5] >> (d & 31)) & 1u);
            }
            put(g, ok, ng);
          }
        } else {
#pragma unroll 4
          for (int g = 0; g < GPW; ++g) {
            const long long v = rd.raw64(q, g);
            bool ok;
            if constexpr (kind == PK_RANGE) ok = pred_test<PT_RANGE>(p, t.aux, v);
            else if constexpr (kind == PK_NE) ok = pred_test<PT_NE>(p, t.aux, v);
            else if constexpr (kind == PK_BITMAP) ok = pred_test<PT_BITMAP>(p, t.aux, v);
            else ok = pred_test<PT_LIST>(p, t.aux, v);
            put(g, ok, ng);
          }
        }
      }
    }
    if constexpr (cl == PC_LAST) {
      pm &= acc;
      acc = 0;
    }
  });
  return pm & valid;
}

// ------------------------------------------------------------------ aggregation
// Digit of key K at tile row o (64-bit: hash domains pack wide digits).
template <class S, int K>
__device__ __forceinline__ bool fast_digit(const QueryDesc& q, const TileView& t, uint32_t o, unsigned long long* d,
                                           long long* raw) {
  constexpr int c = S::kcol(K);
  const KeyDesc& k = q.keys[K];
  uint32_t x;
  if constexpr (S::kn32(K)) {
    const int v = fast_raw32<S, c>(q, t, o);
    *raw = v;
    x = (uint32_t)v - (uint32_t)(int)k.kmin;
    if constexpr (!S::kremap(K)) {
      *d = x;
      return x < k.card;
    }
  } else {
    const long long v = fast_raw<S, c>(q, t, o);
    *raw = v;
    const unsigned long long dd = (unsigned long long)v - (unsigned long long)k.kmin;
    if constexpr (!S::kremap(K)) {
      *d = dd;
      return v >= k.kmin && dd < k.card;
    }
    if (v < k.kmin || dd >= 32ull * k.aux_len) return false;
    x = (uint32_t)dd;
  }
  if constexpr (S::kremap(K)) {
    if (x >= 32u * k.aux_len) return false;
    const uint32_t w = t.aux[k.aux_off + (x >> 5)];
    if (!((w >> (x & 31)) & 1u)) return false;
    *d = t.aux[k.prefix_off + (x >> 5)] + __popc(w & ((1u << (x & 31)) - 1u));
    return true;
  }
  return true;
}

// One aggregate's update of shared slot `slot` (or, when the table had no
// free slot, of the global accumulators at index gid, see gindex).
template <class S, int I>
__device__ __forceinline__ void fast_update(const QueryDesc& q, const Smem& sm, int slot, uint32_t gid, long long v) {
  constexpr int kind = S::akind(I);
  const uint32_t slots = q.table_slots;
  if constexpr (kind == AK_SUM) {
    if (slot >= 0) {
      if constexpr (S::as32(I) == 3)
        split_add(sword32(q, sm, S::asw32(I), slot), sword32(q, sm, S::asw32(I) + 1, slot), (unsigned)v);
      else if constexpr (S::as32(I)) atomicAdd(&sm.tacc32[(size_t)S::asw32(I) * slots + slot], (unsigned)v);
      else if constexpr (!S::awide(I)) smem_add64(&sm.tacc[(size_t)S::asw(I) * slots + slot], v);
      else atomic_add_i128(&sm.tacc[(size_t)S::asw(I) * slots + slot], &sm.tacc[(size_t)(S::asw(I) + 1) * slots + slot],
                           sext(v));
    } else {
      global_add_limbs(gword(q, S::agw(I), gid), gword(q, S::agw(I) + 1, gid), gword(q, S::agw(I) + 2, gid), sext(v));
    }
  } else if constexpr (kind == AK_SUM2) {
    const long long v2 = v * v;   // |v| < 2^31 (planner)
    if (slot >= 0) {
      if constexpr (!S::awide(I)) smem_add64(&sm.tacc[(size_t)S::asw(I) * slots + slot], v2);
      else atomic_add_i128(&sm.tacc[(size_t)S::asw(I) * slots + slot], &sm.tacc[(size_t)(S::asw(I) + 1) * slots + slot],
                           sext(v2));
    } else {
      global_add_limbs(gword(q, S::agw(I), gid), gword(q, S::agw(I) + 1, gid), gword(q, S::agw(I) + 2, gid), sext(v2));
    }
  } else if constexpr (kind == AK_MIN || kind == AK_MAX) {
    constexpr bool mn = kind == AK_MIN;
    if (slot >= 0) {
      if constexpr (S::aw32(I)) {
        int* p = reinterpret_cast<int*>(&sm.tacc32[(size_t)S::asw32(I) * slots + slot]);
        const int cur = *reinterpret_cast<volatile int*>(p);
        if (mn ? (int)v < cur : (int)v > cur) {
          if (mn) atomicMin(p, (int)v);
          else atomicMax(p, (int)v);
        }
      } else {
        long long* p = reinterpret_cast<long long*>(&sm.tacc[(size_t)S::asw(I) * slots + slot]);
        const long long cur = *reinterpret_cast<volatile long long*>(p);
        if (mn ? v < cur : v > cur) {
          if (mn) atomicMin(p, v);
          else atomicMax(p, v);
        }
      }
    } else {
      if (mn) atomicMin(reinterpret_cast<long long*>(gword(q, S::agw(I), gid)), v);
      else atomicMax(reinterpret_cast<long long*>(gword(q, S::agw(I), gid)), v);
    }
  }
}

// Aggregates of an index-encoded column: only listed rows differ from the
// default, which finalize adds back from COUNT.
template <class S, int I>
__device__ __forceinline__ void fast_index_update(const QueryDesc& q, const Smem& sm, const TileView& t, int slot,
                                                  uint32_t gid, uint32_t o) {
  constexpr int kind = S::akind(I);
  const AggDesc& a = q.aggs[I];
  long long v;
  if (!index_lookup(q.cols[S::acol(I)], t, o, &v)) return;
  if constexpr (kind == AK_ISUM) {
    sum_add(q, sm, a, slot, gid, index_delta(v, a.base));
  } else if constexpr (kind == AK_ISUM2) {
    const long long dv = v - a.base;   // |v - default| < 2^31 (planner)
    sum_add(q, sm, a, slot, gid, sext(dv * dv));
  } else {
    minmax_add(q, sm, a, slot, gid, v, kind == AK_IMIN);
    if (slot >= 0) atomicAdd(slisted(q, sm, a, slot), 1u);
    else atomicAdd(gword(q, a.gw + 1, gid), 1ull);
  }
}

// Whether every aggregate of the shape can be reduced across a warp in 32-bit
// arithmetic first (COUNT, SUMs of values below 2^24 in magnitude, MIN / MAX
// of 32-bit values; index-column aggregates cannot).
template <class S>
__device__ constexpr bool seg_reducible() {
  for (int i = 0; i < S::n_aggs; ++i) {
    const int k = S::akind(i);
    if (k == AK_SUM && !S::ared32(i)) return false;
    if ((k == AK_MIN || k == AK_MAX) && !S::aw32(i)) return false;
    if (k == AK_ISUM || k == AK_IMIN || k == AK_IMAX || k == AK_SUM2 || k == AK_ISUM2) return false;
  }
  return true;
}

// Packed prefix sums for runs of equal groups: each SUM aggregate whose
// inputs lie in [0, 2^aub) takes a field of aub + 5 bits (a sum of 32 inputs
// fits) in one of two 32-bit words, in aggregate order.  pk_place gives the
// word (word = true) or the bit offset of aggregate `want`, -1 when the SUMs
// do not all fit.
template <class S>
__device__ constexpr int pk_place(int want, bool word) {
  int w = 0, off = 0;
  for (int i = 0; i < S::n_aggs; ++i) {
    if (S::akind(i) != AK_SUM) continue;
    const int b = S::aub(i);
    if (b == 0) return -1;
    if (off + b + 5 > 32) {
      ++w;
      off = 0;
    }
    if (w > 1) return -1;
    if (i == want) return word ? w : off;
    off += b + 5;
  }
  return -1;
}

template <class S>
__device__ constexpr bool pk_ok() {
  bool any = false;
  for (int i = 0; i < S::n_aggs; ++i)
    if (S::akind(i) == AK_SUM) {
      if (pk_place<S>(i, true) < 0) return false;
      any = true;
    }
  return any;
}

// Aggregate the n_pass compacted rows of this warp, 32 at a time (one per
// lane): group id from the key digits, a shared-table slot, COUNT and every
// aggregate.  A single-group query reduces across the warp first.
//
// Line mode (S::line_mode, tiles with line_ok): key 0 is an RLE column and
// the shared table holds one line per run of it, so "gid" is the slot itself:
// line (run ordinal line_cur + rank, modulo the line count) times the line
// width plus the other keys' packed digits; the flush recovers the group.  A
// tile with more runs than lines (line_ok false) updates the global
// accumulators of the true group directly.
template <class S>
__device__ __forceinline__ void fast_agg_step(const QueryDesc& q, const Smem& sm, const TileView& t, uint32_t o,
                                              bool act, unsigned long long row0, bool line_ok,
                                              unsigned long long line_cur) {
  const int lane = threadIdx.x & 31;
  // the packed key: 64-bit for a hash domain, else the 32-bit dense gid
  typename Pick<S::ghash, unsigned long long, uint32_t>::type gid = 0;
  uint32_t line = 0;
  static_for<S::n_keys>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr (S::line_mode && k == 0) {
      if (line_ok) {
        constexpr int jl = S::bslot(S::kcol(0));
        constexpr uint32_t nw = S::tile_rows / 32;
        const uint32_t r = rank_incl(t.bm + jl * nw, t.pre + jl * (nw + 1), o);
        line = (uint32_t)(line_cur + r) & ((1u << q.line_log2) - 1u);
        return;
      }
    }
    unsigned long long d = 0;
    long long raw = 0;
    if (!fast_digit<S, k>(q, t, o, &d, &raw)) {
      if (act) {
        act = false;
        report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)k << 8), row0 + o, (unsigned long long)raw);
      }
      d = 0;
    }
    if constexpr (S::ghash) gid += d * q.keys[k].stride;
    else gid += (uint32_t)d * (uint32_t)q.keys[k].stride;
  });
  // a line's slots are its inner digits with the low bits XOR-ed by the
  // line, so that rows of equal inner digits in different runs fall in
  // different shared-memory banks
  if constexpr (S::line_mode)
    if (line_ok) gid = line * q.line_inner + (gid ^ (line & q.line_swz));
  long long val[S::n_aggs + 1];
  static_for<S::n_aggs>([&](auto A) {
    constexpr int i = decltype(A)::value;
    constexpr int kind = S::akind(i);
    if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX || kind == AK_SUM2) {
      if constexpr (S::asrc(i) == i) {
        if constexpr (S::an32(i)) val[i] = (long long)fast_raw32<S, S::acol(i)>(q, t, o);
        else val[i] = fast_raw<S, S::acol(i)>(q, t, o);
      } else {
        val[i] = val[S::asrc(i)];
      }
    }
  });
  if constexpr (S::one_group) {
    const uint32_t n = __popc(__ballot_sync(0xFFFFFFFFu, act));
    if (lane == 0) atomicAdd(scount(q, sm, 0), n);
    static_for<S::n_aggs>([&](auto A) {
      constexpr int i = decltype(A)::value;
      constexpr int kind = S::akind(i);
      if constexpr (kind == AK_SUM && S::ared32(i)) {
        const int r = __reduce_add_sync(0xFFFFFFFFu, act ? (int)val[i] : 0);
        if (lane == 0) {
          if constexpr (S::as32(i) == 3)
            split_add(sword32(q, sm, S::asw32(i), 0), sword32(q, sm, S::asw32(i) + 1, 0), (unsigned)r);
          else if constexpr (S::as32(i)) atomicAdd(&sm.tacc32[(size_t)S::asw32(i) * q.table_slots], (unsigned)r);
          else smem_add64(&sm.tacc[(size_t)S::asw(i) * q.table_slots], (long long)r);
        }
      } else if constexpr ((kind == AK_MIN || kind == AK_MAX) && S::aw32(i)) {
        constexpr bool mn = kind == AK_MIN;
        const int x = act ? (int)val[i] : (mn ? INT_MAX : INT_MIN);
        const int r = mn ? __reduce_min_sync(0xFFFFFFFFu, x) : __reduce_max_sync(0xFFFFFFFFu, x);
        if (lane == 0) {
          int* p = reinterpret_cast<int*>(&sm.tacc32[(size_t)S::asw32(i) * q.table_slots]);
          if (mn) atomicMin(p, r);
          else atomicMax(p, r);
        }
      } else if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX || kind == AK_SUM2) {
        if (act) fast_update<S, i>(q, sm, 0, 0, val[i]);
      } else if constexpr (kind != AK_COUNT) {
        if (act) fast_index_update<S, i>(q, sm, t, 0, 0, o);
      }
    });
  } else {
    if constexpr (seg_reducible<S>()) {
      // Sorted keys (runs of equal groups among consecutive passing rows):
      // reduce each run of equal gids across the warp first and let its
      // last lane update the table once -- COUNT = run length, SUM and
      // MIN / MAX by a segmented shuffle scan.  Taken when the runs average
      // two or more rows; otherwise every lane updates (below).
      const auto prev = __shfl_up_sync(0xFFFFFFFFu, gid, 1);
      const uint32_t actm = __ballot_sync(0xFFFFFFFFu, act);
      // (a head also follows a lane without a row: in-place groups have holes)
      const bool head = act && (lane == 0 || prev != gid || !((actm >> (lane - 1)) & 1u));
      const uint32_t heads = __ballot_sync(0xFFFFFFFFu, head);
      if (2 * __popc(heads) <= __popc(actm)) {
        const uint32_t upto = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
        const int seg0 = 31 - __clz(heads & upto);   // first lane of my run (act lanes)
        const bool tail = act && (lane == 31 || !((actm >> (lane + 1)) & 1u) || ((heads >> (lane + 1)) & 1u));
        int red[S::n_aggs + 1];
        constexpr bool packed = pk_ok<S>();
        if constexpr (packed) {
          // every SUM at once: an inclusive prefix scan of the packed
          // fields, a run's sum the difference at its ends (fields never
          // carry into each other)
          uint32_t pw0 = 0, pw1 = 0;
          static_for<S::n_aggs>([&](auto A) {
            constexpr int i = decltype(A)::value;
            if constexpr (S::akind(i) == AK_SUM) {
              const uint32_t x = act ? ((uint32_t)val[i] << pk_place<S>(i, false)) : 0u;
              if constexpr (pk_place<S>(i, true) == 0) pw0 += x;
              else pw1 += x;
            }
          });
          constexpr bool two = [] {
            for (int i = 0; i < S::n_aggs; ++i)
              if (S::akind(i) == AK_SUM && pk_place<S>(i, true) == 1) return true;
            return false;
          }();
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y0 = __shfl_up_sync(0xFFFFFFFFu, pw0, d);
            if (lane >= d) pw0 += y0;
            if constexpr (two) {
              const uint32_t y1 = __shfl_up_sync(0xFFFFFFFFu, pw1, d);
              if (lane >= d) pw1 += y1;
            }
          }
          const int src = seg0 > 0 ? seg0 - 1 : 0;
          uint32_t b0 = __shfl_sync(0xFFFFFFFFu, pw0, src), b1 = 0;
          if constexpr (two) b1 = __shfl_sync(0xFFFFFFFFu, pw1, src);
          if (seg0 == 0) b0 = b1 = 0;
          static_for<S::n_aggs>([&](auto A) {
            constexpr int i = decltype(A)::value;
            if constexpr (S::akind(i) == AK_SUM) {
              constexpr int off = pk_place<S>(i, false), width = S::aub(i) + 5;
              const uint32_t dw = pk_place<S>(i, true) == 0 ? pw0 - b0 : pw1 - b1;
              red[i] = (int)((dw >> off) & (width >= 32 ? 0xFFFFFFFFu : ((1u << width) - 1u)));
            }
          });
        }
        static_for<S::n_aggs>([&](auto A) {
          constexpr int i = decltype(A)::value;
          constexpr int kind = S::akind(i);
          if constexpr ((kind == AK_SUM && !packed) || kind == AK_MIN || kind == AK_MAX) {
            constexpr bool mn = kind == AK_MIN;
            int x = act ? (int)val[i] : (kind == AK_SUM ? 0 : (mn ? INT_MAX : INT_MIN));
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
              if (lane - d >= seg0) x = kind == AK_SUM ? x + y : (mn ? min(x, y) : max(x, y));
            }
            red[i] = x;
          }
        });
        if (tail) {
          int slot = -1;
          uint32_t gi = 0;
          bool ok = true;
          const unsigned cnt = (unsigned)(lane - seg0 + 1);
          if constexpr (S::table_dense) slot = (int)gid;
          else if constexpr (S::line_mode) slot = line_ok ? (int)gid : -1;
          else slot = table_slot_t<S::ghash>(q, sm, gid);
          if (slot >= 0) {
            atomicAdd(scount(q, sm, slot), cnt);
          } else {
            const long long g = gindex_t<S::ghash>(q, gid);
            ok = g >= 0;
            gi = (uint32_t)g;
            if (ok) atomicAdd(gword(q, 0, gi), (unsigned long long)cnt);
          }
          static_for<S::n_aggs>([&](auto A) {
            constexpr int i = decltype(A)::value;
            constexpr int kind = S::akind(i);
            if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX) {
              if (ok) fast_update<S, i>(q, sm, slot, gi, (long long)red[i]);
            }
          });
        }
        return;
      }
    }
    int slot = -1;
    uint32_t gi = 0;   // global accumulator index, used when the shared table has no slot
    if (act) {
      if constexpr (S::table_dense) slot = (int)gid;
      else if constexpr (S::line_mode) slot = line_ok ? (int)gid : -1;
      else slot = table_slot_t<S::ghash>(q, sm, gid);
      if (slot >= 0) {
        atomicAdd(scount(q, sm, slot), 1u);
      } else {
        const long long g = gindex_t<S::ghash>(q, gid);
        if (g < 0) act = false;   // global hash table full: the host retries larger
        gi = (uint32_t)g;
        if (act) atomicAdd(gword(q, 0, gi), 1ull);
      }
    }
    static_for<S::n_aggs>([&](auto A) {
      constexpr int i = decltype(A)::value;
      constexpr int kind = S::akind(i);
      if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX || kind == AK_SUM2) {
        if (act) fast_update<S, i>(q, sm, slot, gi, val[i]);
      } else if constexpr (kind != AK_COUNT) {
        if (act) fast_index_update<S, i>(q, sm, t, slot, gi, o);
      }
    });
  }
}

// The compacted rows list[0 .. n_pass), 32 at a time.
template <class S>
__device__ __forceinline__ void fast_aggregate(const QueryDesc& q, const Smem& sm, const TileView& t,
                                               const uint16_t* list, uint32_t n_pass, unsigned long long row0,
                                               bool line_ok, unsigned long long line_cur) {
  const int lane = threadIdx.x & 31;
  for (uint32_t j0 = 0; j0 < n_pass; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool act = j < n_pass;
    fast_agg_step<S>(q, sm, t, list[act ? j : j0], act, row0, line_ok, line_cur);
  }
}

// ------------------------------------------------------------------ helper warp
// Bits per row of a staged column.
template <class S, int C>
__device__ __forceinline__ constexpr uint32_t col_bits() {
  return S::enc(C) == ENC_PLAIN ? (S::v64(C) ? 64u : 32u) : (uint32_t)S::bw(C);
}

// A predicate on one run / listed value (the helper's once-per-value test),
// complemented when the predicate is negated.
template <class S, int I>
__device__ __forceinline__ bool fast_pred_value(const QueryDesc& q, const uint32_t* aux, long long v) {
  constexpr int kind = S::pkind(I);
  const PredDesc& p = q.preds[I];
  bool r;
  if constexpr (kind == PK_RANGE) r = pred_test<PT_RANGE>(p, aux, v);
  else if constexpr (kind == PK_NE) r = pred_test<PT_NE>(p, aux, v);
  else if constexpr (kind == PK_BITMAP) r = pred_test<PT_BITMAP>(p, aux, v);
  else if constexpr (kind == PK_LIST) r = pred_test<PT_LIST>(p, aux, v);
  else r = kind == PK_TRUE;
  return r != S::pneg(I);
}

// Line mode: the flush of one shared slot with the shape's aggregates known
// at compile time (the generic flush_slot and reset_slot read them from the
// descriptor): add slot s (cnt rows) into group gid's global accumulators,
// then clear it.
template <class S>
__device__ __forceinline__ void fast_flush_slot(const QueryDesc& q, const Smem& sm, uint32_t s, unsigned cnt,
                                                uint32_t gid) {
  atomicAdd(gword(q, 0, gid), (unsigned long long)cnt);
  *scount(q, sm, s) = 0;
  static_for<S::n_aggs>([&](auto A) {
    constexpr int i = decltype(A)::value;
    constexpr int kind = S::akind(i);
    if constexpr (kind == AK_SUM || kind == AK_ISUM || kind == AK_SUM2 || kind == AK_ISUM2) {
      I128 x;
      if constexpr (S::as32(i) == 3) {
        x = sext(split_value(sword32(q, sm, S::asw32(i), s), sword32(q, sm, S::asw32(i) + 1, s)));
        *sword32(q, sm, S::asw32(i), s) = 0;
        *sword32(q, sm, S::asw32(i) + 1, s) = 0;
      } else if constexpr (S::as32(i) == 1) {
        x = sext((long long)(unsigned)*sword32(q, sm, S::asw32(i), s));
        *sword32(q, sm, S::asw32(i), s) = 0;
      } else if constexpr (S::as32(i) == 2) {
        x = sext((long long)*sword32(q, sm, S::asw32(i), s));
        *sword32(q, sm, S::asw32(i), s) = 0;
      } else if constexpr (S::awide(i)) {
        x.lo = *sword(q, sm, S::asw(i), s);
        x.hi = (long long)*sword(q, sm, S::asw(i) + 1, s);
        *sword(q, sm, S::asw(i), s) = 0;
        *sword(q, sm, S::asw(i) + 1, s) = 0;
      } else {
        x = sext((long long)*sword(q, sm, S::asw(i), s));
        *sword(q, sm, S::asw(i), s) = 0;
      }
      global_add_limbs(gword(q, S::agw(i), gid), gword(q, S::agw(i) + 1, gid), gword(q, S::agw(i) + 2, gid), x);
    } else if constexpr (kind == AK_MIN || kind == AK_MAX || kind == AK_IMIN || kind == AK_IMAX) {
      constexpr bool mn = kind == AK_MIN || kind == AK_IMIN;
      long long v;
      if constexpr (S::aw32(i)) {
        v = *sword32(q, sm, S::asw32(i), s);
        *sword32(q, sm, S::asw32(i), s) = mn ? INT_MAX : INT_MIN;
        if (v != (mn ? (long long)INT_MAX : (long long)INT_MIN)) {
          if (mn) atomicMin(reinterpret_cast<long long*>(gword(q, S::agw(i), gid)), v);
          else atomicMax(reinterpret_cast<long long*>(gword(q, S::agw(i), gid)), v);
        }
      } else {
        v = (long long)*sword(q, sm, S::asw(i), s);
        *sword(q, sm, S::asw(i), s) = mn ? (unsigned long long)LLONG_MAX : (unsigned long long)LLONG_MIN;
        if (v != (mn ? LLONG_MAX : LLONG_MIN)) {
          if (mn) atomicMin(reinterpret_cast<long long*>(gword(q, S::agw(i), gid)), v);
          else atomicMax(reinterpret_cast<long long*>(gword(q, S::agw(i), gid)), v);
        }
      }
      if constexpr (kind == AK_IMIN || kind == AK_IMAX) {
        unsigned* lc = reinterpret_cast<unsigned*>(sword32(q, sm, S::asw32(i) + (S::aw32(i) ? 1 : 0), s));
        if (*lc) atomicAdd(gword(q, S::agw(i) + 1, gid), (unsigned long long)*lc);
        *lc = 0;
      }
    }
  });
}

// Line mode: flush the lines of runs [ord_lo, ord_hi), which have all ended,
// while the other warps still aggregate; the lines' slots are dealt to the
// compute threads (thread `me` of `threads`).  No run being aggregated
// shares a line with these (the tile walk's full-flush rule).
template <class S>
__device__ __forceinline__ void fast_flush_lines(const QueryDesc& q, const Smem& sm, unsigned long long ord_lo,
                                                 unsigned long long ord_hi, uint32_t me, uint32_t threads) {
  const uint32_t lines = 1u << q.line_log2;
  const uint32_t inner = q.line_inner;
  const uint32_t n = (uint32_t)(ord_hi - ord_lo) * inner;   // at most lines * inner slots
  for (uint32_t f = me; f < n; f += threads) {
    const uint32_t xi = f / inner;
    const uint32_t j = f - xi * inner;
    const uint32_t line = (uint32_t)(ord_lo + xi) & (lines - 1u);
    const uint32_t s = line * inner + j;
    const unsigned cnt = *scount(q, sm, s);
    if (cnt == 0) continue;
    const unsigned long long d = sm.tkeys64[line];
    const unsigned long long gid = d * q.keys[0].stride + (j ^ (line & q.line_swz));
    if (d == ~0ull || gid >= q.n_groups) {
      report(q, CQ_ERR_INVALID_ARG, 4ull, s, gid);
      reset_slot(q, sm, s);
      continue;
    }
    fast_flush_slot<S>(q, sm, s, cnt, (uint32_t)gid);
  }
}

// ------------------------------------------------------------------ serial segments
// Sorted data (Section 7: an aggregate over a run of equal groups is one
// update).  Every lane walks R consecutive rows of its own from registers,
// keeps the open stretch's group, COUNT and partial aggregates, and updates
// the group table once per stretch of passing rows with one group: no
// compaction, no shuffles, no per-row table access.  Taken when the filter
// is decided by pass bitmaps alone, every key but the run-line key and every
// aggregated value is a field of at most 32 bits of a staged column, and
// every aggregate reduces in 32 bits.

template <class S>
__device__ constexpr int col_bits_of(int c) {
  return S::enc(c) == ENC_PLAIN ? (S::v64(c) ? 64 : 32) : S::bw(c);
}

template <class S>
__device__ constexpr bool staged32(int c) {
  return ((S::enc(c) == ENC_PLAIN && !S::v64(c)) || S::enc(c) == ENC_PACKED || S::enc(c) == ENC_DICT) &&
         col_bits_of<S>(c) <= 32;
}

// Index of column c among the staged columns (-1: not staged).
template <class S>
__device__ constexpr int ser_rc(int c) {
  for (int i = 0; i < S::n_row_cols; ++i)
    if (S::row_col(i) == c) return i;
  return -1;
}

// Rows a lane walks: the smallest of 8, 16, 32 at which every staged
// column's fields end on a 32-bit word boundary.
template <class S>
__device__ constexpr int ser_rows() {
  int r = 8;
  for (int i = 0; i < S::n_row_cols; ++i)
    while ((r * col_bits_of<S>(S::row_col(i))) % 32 != 0) r *= 2;
  return r;
}

template <class S>
__device__ constexpr bool ser_ok() {
  if (!seg_reducible<S>() || S::one_group || S::ghash) return false;
  for (int i = 0; i < S::n_preds; ++i)
    if (S::ppbm(i) == 0xFF && S::pkind(i) != PK_TRUE && S::pkind(i) != PK_FALSE) return false;
  for (int k = 0; k < S::n_keys; ++k) {
    if (S::line_mode && k == 0) continue;
    if (!staged32<S>(S::kcol(k)) || ser_rc<S>(S::kcol(k)) < 0 || !S::kn32(k)) return false;
  }
  for (int i = 0; i < S::n_aggs; ++i) {
    const int kind = S::akind(i);
    if (kind == AK_COUNT) continue;
    if (kind != AK_SUM && kind != AK_MIN && kind != AK_MAX) return false;
    if (!staged32<S>(S::acol(i)) || ser_rc<S>(S::acol(i)) < 0 || !S::an32(i)) return false;
  }
  for (int i = 0; i < S::n_row_cols; ++i)
    if (col_bits_of<S>(S::row_col(i)) > 32) return false;
  return true;
}

// Field r (a constant) of B-bit fields held in registers, LSB first.
template <int B, int r, int N>
__device__ __forceinline__ uint32_t ser_field(const uint32_t (&w)[N]) {
  constexpr int bit = r * B, wi = bit >> 5, sh = bit & 31;
  if constexpr (B == 32) return w[wi];
  else if constexpr (sh + B <= 32) return (w[wi] >> sh) & ((1u << B) - 1u);
  else return __funnelshift_r(w[wi], w[wi + 1], sh) & ((1u << B) - 1u);
}

// Digit of key K from its 32-bit raw value (as fast_digit).
template <class S, int K>
__device__ __forceinline__ bool ser_digit(const QueryDesc& q, const TileView& t, int v, uint32_t* d) {
  const KeyDesc& k = q.keys[K];
  const uint32_t x = (uint32_t)v - (uint32_t)(int)k.kmin;
  if constexpr (!S::kremap(K)) {
    *d = x;
    return x < k.card;
  } else {
    if (x >= 32u * k.aux_len) return false;
    const uint32_t w = t.aux[k.aux_off + (x >> 5)];
    if (!((w >> (x & 31)) & 1u)) return false;
    *d = t.aux[k.prefix_off + (x >> 5)] + __popc(w & ((1u << (x & 31)) - 1u));
    return true;
  }
}

// One stretch's update: cnt rows of group gid, partial aggregates acc.
template <class S>
__device__ __forceinline__ void ser_flush(const QueryDesc& q, const Smem& sm, uint32_t gid, uint32_t cnt,
                                          const int* acc) {
  int slot;
  uint32_t gi = 0;
  bool ok = true;
  if constexpr (S::table_dense || S::line_mode) slot = (int)gid;
  else slot = table_slot_t<false>(q, sm, gid);
  if (slot >= 0) {
    atomicAdd(scount(q, sm, slot), cnt);
  } else {
    const long long g = gindex_t<false>(q, gid);
    ok = g >= 0;
    gi = (uint32_t)g;
    if (ok) atomicAdd(gword(q, 0, gi), (unsigned long long)cnt);
  }
  static_for<S::n_aggs>([&](auto A) {
    constexpr int i = decltype(A)::value;
    constexpr int kind = S::akind(i);
    if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX)
      if (ok) fast_update<S, i>(q, sm, slot, gi, (long long)acc[i]);
  });
}

// Shared-memory reductions issued under a predicate (no branch): the walk
// issues its stretch update on every row, live only where a stretch ends.
__device__ __forceinline__ void red_add_if(bool p, const void* a, unsigned v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q red.shared.add.u32 [%0], %1;\n}"
               ::"r"(smem_addr(a)), "r"(v), "r"((unsigned)p) : "memory");
}
__device__ __forceinline__ void red_min_if(bool p, const void* a, int v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q red.shared.min.s32 [%0], %1;\n}"
               ::"r"(smem_addr(a)), "r"(v), "r"((unsigned)p) : "memory");
}
__device__ __forceinline__ void red_max_if(bool p, const void* a, int v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q red.shared.max.s32 [%0], %1;\n}"
               ::"r"(smem_addr(a)), "r"(v), "r"((unsigned)p) : "memory");
}

// Whether the stretch update can be issued that way: slots are group ids
// (run lines or a dense table) and every accumulator is a 32-bit word
// updated without its old value (COUNT, 32-bit or split-limb SUMs, 32-bit
// MIN / MAX).
template <class S>
__device__ constexpr bool ser_pred_ok() {
  if (!(S::line_mode || S::table_dense)) return false;
  for (int i = 0; i < S::n_aggs; ++i) {
    const int kind = S::akind(i);
    if (kind == AK_SUM && S::as32(i) == 0) return false;
    if ((kind == AK_MIN || kind == AK_MAX) && !S::aw32(i)) return false;
  }
  return true;
}

// ser_flush under predicate f (slot = gid; gid need not be a slot when f is
// false: no address is touched then).
template <class S>
__device__ __forceinline__ void ser_flush_if(const QueryDesc& q, const Smem& sm, bool f, uint32_t gid,
                                             uint32_t cnt, const int* acc) {
  const int slot = (int)gid;
  red_add_if(f, scount(q, sm, slot), cnt);
  static_for<S::n_aggs>([&](auto A) {
    constexpr int i = decltype(A)::value;
    constexpr int kind = S::akind(i);
    if constexpr (kind == AK_SUM) {
      if constexpr (S::as32(i) == 3) {
        const unsigned x = (unsigned)acc[i];
        red_add_if(f, sword32(q, sm, S::asw32(i), slot), x & ((1u << kSplitBits) - 1u));
        red_add_if(f && (x >> kSplitBits) != 0u, sword32(q, sm, S::asw32(i) + 1, slot), x >> kSplitBits);
      } else {
        red_add_if(f, sword32(q, sm, S::asw32(i), slot), (unsigned)acc[i]);
      }
    } else if constexpr (kind == AK_MIN) {
      red_min_if(f, sword32(q, sm, S::asw32(i), slot), acc[i]);
    } else if constexpr (kind == AK_MAX) {
      red_max_if(f, sword32(q, sm, S::asw32(i), slot), acc[i]);
    }
  });
}

// Rows o0 .. o0 + R - 1 of one lane: `pass` their filter bits, `starts` the
// run-start bits of key 0's column from row o0 on (VARY: a run starts
// inside, so the line advances), `line` the line at row o0.  Without CHECK
// every field of every staged key is a valid digit (ser_keys_total), so the
// digits are not tested.
template <class S, int R, bool VARY, bool CHECK>
__device__ __forceinline__ void ser_walk(const QueryDesc& q, const Smem& sm, const TileView& t, uint32_t o0,
                                         uint32_t pass, uint32_t starts, uint32_t line, unsigned long long row0) {
  constexpr int NRC = S::n_row_cols > 0 ? S::n_row_cols : 1;
  uint32_t w[NRC][R];
  static_for<S::n_row_cols>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int NW = R * col_bits_of<S>(S::row_col(i)) / 32;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(t.stage + S::stage_off(S::row_col(i))) + (o0 / R) * NW;
    if constexpr (NW % 4 == 0) {
#pragma unroll
      for (int j = 0; j < NW / 4; ++j) {
        const uint4 v = reinterpret_cast<const uint4*>(src)[j];
        w[i][4 * j] = v.x;
        w[i][4 * j + 1] = v.y;
        w[i][4 * j + 2] = v.z;
        w[i][4 * j + 3] = v.w;
      }
    } else if constexpr (NW % 2 == 0) {
#pragma unroll
      for (int j = 0; j < NW / 2; ++j) {
        const uint2 v = reinterpret_cast<const uint2*>(src)[j];
        w[i][2 * j] = v.x;
        w[i][2 * j + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j) w[i][j] = src[j];
    }
  });
  uint32_t lmask = 0;
  if constexpr (S::line_mode) lmask = (1u << q.line_log2) - 1u;
  // A failing row's group is kNone, so a stretch ends exactly where the
  // group changes; a failing stretch accumulates too but is never flushed.
  constexpr uint32_t kNone = 0xFFFFFFFFu;   // above every group id (< 2^32 - 1)
  uint32_t cur = kNone, s0 = 0;   // the open stretch's group and first row
  int acc[S::n_aggs + 1];
#pragma unroll
  for (int i = 0; i <= S::n_aggs; ++i) acc[i] = 0;
  static_for<R>([&](auto RI) {
    constexpr int r = decltype(RI)::value;
    if constexpr (VARY && r > 0) line = (line + ((starts >> r) & 1u)) & lmask;
    bool p = (pass >> r) & 1u;
    uint32_t g = 0;
    static_for<S::n_keys>([&](auto K) {
      constexpr int k = decltype(K)::value;
      if constexpr (!(S::line_mode && k == 0)) {
        constexpr int c = S::kcol(k);
        const int v = (int)ser_field<col_bits_of<S>(c), r>(w[ser_rc<S>(c)]);
        uint32_t d;
        if constexpr (CHECK) {
          if (!ser_digit<S, k>(q, t, v, &d)) {
            if (p) {
              report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)k << 8), row0 + o0 + r,
                     (unsigned long long)(long long)v);
              p = false;
            }
            d = 0;
          }
        } else {
          d = (uint32_t)v;   // (digit = field: the key's minimum is 0)
        }
        g += d * (uint32_t)q.keys[k].stride;
      }
    });
    if constexpr (S::line_mode) g = line * q.line_inner + (g ^ (line & q.line_swz));
    g = p ? g : kNone;
    if constexpr (r == 0) {
      cur = g;
      static_for<S::n_aggs>([&](auto A) {
        constexpr int i = decltype(A)::value;
        constexpr int kind = S::akind(i);
        if constexpr (kind == AK_MIN || kind == AK_MAX) acc[i] = kind == AK_MIN ? INT_MAX : INT_MIN;
      });
    } else if constexpr (ser_pred_ok<S>()) {
      // the stretch before this row ends where the group changes: its update
      // is issued on every row, live only there
      const bool brk = g != cur;
      ser_flush_if<S>(q, sm, brk && cur != kNone, cur, (uint32_t)r - s0, acc);
      cur = g;
      s0 = brk ? (uint32_t)r : s0;
      static_for<S::n_aggs>([&](auto A) {
        constexpr int i = decltype(A)::value;
        constexpr int kind = S::akind(i);
        if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX)
          acc[i] = brk ? (kind == AK_SUM ? 0 : (kind == AK_MIN ? INT_MAX : INT_MIN)) : acc[i];
      });
    } else if (g != cur) {
      // the stretch before this row ends
      if (cur != kNone) ser_flush<S>(q, sm, cur, (uint32_t)r - s0, acc);
      cur = g;
      s0 = r;
      static_for<S::n_aggs>([&](auto A) {
        constexpr int i = decltype(A)::value;
        constexpr int kind = S::akind(i);
        if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX)
          acc[i] = kind == AK_SUM ? 0 : (kind == AK_MIN ? INT_MAX : INT_MIN);
      });
    }
    static_for<S::n_aggs>([&](auto A) {
      constexpr int i = decltype(A)::value;
      constexpr int kind = S::akind(i);
      if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX) {
        constexpr int c = S::acol(i);
        const int v = (int)ser_field<col_bits_of<S>(c), r>(w[ser_rc<S>(c)]);
        acc[i] = kind == AK_SUM ? acc[i] + v : (kind == AK_MIN ? min(acc[i], v) : max(acc[i], v));
      }
    });
  });
  if (cur != kNone) ser_flush<S>(q, sm, cur, (uint32_t)R - s0, acc);
}

// Whether every field of every staged key is a valid digit: no remap, key
// minimum 0 and at least 2^B digit values for B-bit fields.
template <class S>
__device__ __forceinline__ bool ser_keys_total(const QueryDesc& q) {
  bool all = true;
  static_for<S::n_keys>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr (!(S::line_mode && k == 0)) {
      constexpr int B = col_bits_of<S>(S::kcol(k));
      if constexpr (S::kremap(k) || B >= 32) all = false;
      else all = all && q.keys[k].kmin == 0 && q.keys[k].card >= (1ull << B);
    }
  });
  return all;
}

// The compute warps' serial pass over a tile: the tile's passes of 32 * R
// consecutive rows (lane l takes rows l * R .. l * R + R - 1 of a pass, so
// that the lanes' staged words are consecutive in shared memory) are dealt
// to the warps from a shared counter, one per tile parity, so that warps
// whose rows pass more take fewer passes.  Thread 0 clears the next tile's
// counter (misc[4 + parity]) at the start of every tile.
template <class S, int NCW, int GPW>
__device__ __forceinline__ void fast_serial(const QueryDesc& q, const Smem& sm, const TileView& t, uint32_t rows,
                                            unsigned long long row0, unsigned long long line_cur) {
  constexpr int R = ser_rows<S>();
  constexpr uint32_t passes = S::tile_rows / (32u * R);
  constexpr uint32_t nw = S::tile_rows / 32;
  constexpr uint32_t inner_bits = R == 32 ? 0xFFFFFFFEu : ((1u << R) - 2u);
  const int lane = threadIdx.x & 31;
  int* ctr = sm.misc + 4 + ((uint32_t)(row0 / S::tile_rows) & 1u);
  for (;;) {
    uint32_t j = 0;
    if (lane == 0) j = (uint32_t)atomicAdd(ctr, 1);
    j = __shfl_sync(0xFFFFFFFFu, j, 0);
    if (j >= passes) break;
    const uint32_t o0 = j * 32u * R + (uint32_t)lane * R;
    uint32_t pass = 0;
    if (o0 < rows) {
      uint32_t valid = R == 32 ? 0xFFFFFFFFu : ((1u << R) - 1u);
      if (rows - o0 < (uint32_t)R) valid &= (1u << (rows - o0)) - 1u;
      // the filter's clauses over the pass-bitmap words of these rows
      uint32_t pm = valid, acc = 0;
      static_for<S::n_preds>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int kind = S::pkind(i);
        constexpr int cl = S::pcl(i);
        if constexpr (S::ppbm(i) != 0xFF) {
          const uint32_t x = t.pbm[(size_t)S::ppbm(i) * nw + (o0 >> 5)] >> (o0 & 31);
          if constexpr (cl == PC_ALONE) pm &= x;
          else acc |= x;
        } else if constexpr (kind == PK_FALSE) {
          if constexpr (cl == PC_ALONE) pm = 0;
        } else if constexpr (kind == PK_TRUE) {
          if constexpr (cl != PC_ALONE) acc = ~0u;
        }
        if constexpr (cl == PC_LAST) {
          pm &= acc;
          acc = 0;
        }
      });
      pass = pm & valid;
    }
    if (!__any_sync(0xFFFFFFFFu, pass != 0)) continue;
    uint32_t line = 0, starts = 0;
    bool vary = false;
    if constexpr (S::line_mode) {
      constexpr int jl = S::bslot(S::kcol(0));
      const uint32_t* B = t.bm + jl * nw;
      const uint32_t oo = o0 < rows ? o0 : 0u;
      line = (uint32_t)(line_cur + rank_incl(B, t.pre + jl * (nw + 1), oo)) & ((1u << q.line_log2) - 1u);
      starts = B[oo >> 5] >> (oo & 31);
      vary = __any_sync(0xFFFFFFFFu, pass != 0 && (starts & inner_bits) != 0);
    }
    if (pass != 0) {
      if (ser_keys_total<S>(q)) {
        if (vary) ser_walk<S, R, true, false>(q, sm, t, o0, pass, starts, line, row0);
        else ser_walk<S, R, false, false>(q, sm, t, o0, pass, starts, line, row0);
      } else {
        if (vary) ser_walk<S, R, true, true>(q, sm, t, o0, pass, starts, line, row0);
        else ser_walk<S, R, false, true>(q, sm, t, o0, pass, starts, line, row0);
      }
    }
  }
}

template <class S>
struct FastBody {
  template <int NCW, int GPW>
  __device__ static __forceinline__ void tile(const QueryDesc& q, const Smem& sm, const TileView& tv, uint32_t wbase,
                                              uint32_t rows, uint16_t* list, unsigned long long row0) {
    constexpr uint32_t GS = NCW * 32;
    // the serial walk's pass counter of the next tile (see fast_serial)
    if constexpr (ser_ok<S>())
      if (threadIdx.x == 0) sm.misc[4 + (((uint32_t)(row0 / S::tile_rows) & 1u) ^ 1u)] = 0;
    bool line_ok = false;
    unsigned long long line_cur = 0;
    if constexpr (S::line_mode) {
      // the tile's runs of key 0's column: ordinals line_cur .. line_cur + nset
      constexpr int jl = S::bslot(S::kcol(0));
      constexpr uint32_t nw = S::tile_rows / 32;
      line_cur = tv.cur[jl];
      const uint32_t nset = tv.pre[jl * (nw + 1) + nw];
      line_ok = nset < (1u << q.line_log2);
      if (line_ok && wbase == 0) line_digits(q, sm, tv, line_cur, nset);
    }
    if constexpr (ser_ok<S>()) {
      // (the same choice in every warp: line_ok is the tile's)
      if (!S::line_mode || line_ok) {
        fast_serial<S, NCW, GPW>(q, sm, tv, rows, row0, line_cur);
        if constexpr (S::line_mode)
          fast_flush_lines<S>(q, sm, tv.line_base, line_cur, threadIdx.x, NCW * 32);
        return;
      }
    }
    const uint32_t pm = fast_filter<S, GS, GPW>(q, tv, wbase, rows);
    bool in_place = false;
    if constexpr (seg_reducible<S>() && !S::one_group) {
      // passing rows in long stretches (sorted data): when at least half of
      // the warp's non-empty 32-row groups pass whole, aggregate the groups
      // in place (lane = row), without compaction
      uint32_t full = 0, busy = 0;
#pragma unroll
      for (int g = 0; g < GPW; ++g) {
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (pm >> g) & 1u);
        full += bal == 0xFFFFFFFFu ? 1u : 0u;
        busy += bal != 0u ? 1u : 0u;
      }
      in_place = busy != 0 && 2 * full >= busy;
      if (in_place) {
        const int lane = threadIdx.x & 31;
        for (int g = 0; g < GPW; ++g) {
          const bool ok = (pm >> g) & 1u;
          if (__ballot_sync(0xFFFFFFFFu, ok))
            fast_agg_step<S>(q, sm, tv, wbase + g * GS + lane, ok, row0, line_ok, line_cur);
        }
      }
    }
    if (!in_place) {
      const uint32_t n_pass = compact<GPW>(pm, wbase, GS, list);
      fast_aggregate<S>(q, sm, tv, list, n_pass, row0, line_ok, line_cur);
    }
    // the lines of the runs that ended before this tile
    if constexpr (S::line_mode)
      fast_flush_lines<S>(q, sm, tv.line_base, line_cur, threadIdx.x, NCW * 32);
  }

  // Bulk copies of tile u's row-level columns into stage st (a full tile's
  // byte counts are constants).
  __device__ static __forceinline__ void issue(const QueryDesc& q, const Smem& sm, unsigned long long u, uint32_t st) {
    constexpr uint32_t T = S::tile_rows;
    uint8_t* dst = sm.stage + (size_t)st * S::stage_bytes;
    const unsigned long long r0 = u * T;
    const bool full = q.n_rows - r0 >= T;
    const uint32_t rows = full ? T : (uint32_t)(q.n_rows - r0);
    uint32_t total = 0;
    static_for<S::n_row_cols>([&](auto I) {
      constexpr int c = S::row_col(decltype(I)::value);
      constexpr uint32_t bits = col_bits<S, c>();
      constexpr uint32_t full_bytes = ((T * bits + 7) / 8 + 15) / 16 * 16;
      total += full ? full_bytes : ((rows * bits + 7) / 8 + 15) / 16 * 16;
    });
    mbar_arrive_expect_tx(&sm.mbar[st], total);
    static_for<S::n_row_cols>([&](auto I) {
      constexpr int c = S::row_col(decltype(I)::value);
      constexpr uint32_t bits = col_bits<S, c>();
      constexpr uint32_t full_bytes = ((T * bits + 7) / 8 + 15) / 16 * 16;
      const uint32_t bytes = full ? full_bytes : ((rows * bits + 7) / 8 + 15) / 16 * 16;
      bulk_g2s(dst + S::stage_off(c), reinterpret_cast<const uint8_t*>(q.cols[c].vals) + r0 * bits / 8, bytes,
               &sm.mbar[st]);
    });
  }

  // Windows of kWin run ends / positions and their values per bitmap column,
  // from the helper cursors on, into window set wb.
  // (helper warp hw of nh takes the columns j with j % nh == hw)
  __device__ static __forceinline__ void prefetch(const QueryDesc& q, const Smem& sm, int wb, int hw, int nh) {
    const int lane = threadIdx.x & 31;
    const unsigned long long* hcur = helper_cursor(sm);
    static_for<S::n_bitmaps>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int c = S::bcol(j);
      if (j % nh != hw) return;
      const ColDesc& cd = q.cols[c];
      const unsigned long long cur = hcur[j];
      const uint32_t avail = cur < cd.n ? (uint32_t)((cd.n - cur) < kWin ? (cd.n - cur) : kWin) : 0u;
      uint8_t* dst = sm.win + ((size_t)wb * S::n_bitmaps + j) * kWin * 16;
      uint8_t* vdst = dst + kWin * 8;
      for (uint32_t i = lane; i < avail; i += 32) {
        if constexpr (S::e64(c)) cp_async8(dst + 8 * i, reinterpret_cast<const long long*>(cd.ends) + cur + i);
        else cp_async4(dst + 4 * i, reinterpret_cast<const int*>(cd.ends) + cur + i);
        if constexpr (S::v64(c)) cp_async8(vdst + 8 * i, reinterpret_cast<const long long*>(cd.vals) + cur + i);
        else cp_async4(vdst + 4 * i, reinterpret_cast<const int*>(cd.vals) + cur + i);
      }
      if (lane == 0) sm.wcnt[wb * kMaxBitmapCols + j] = avail;
    });
    cp_async_commit();
  }

  // Bitmaps (bit o: a run of the column ends at tile row o / row o is listed)
  // with word prefix popcounts, start cursors, and the pass bitmaps of the
  // run-column predicates, for tile [s, e) into buffer buf.
  __device__ static __forceinline__ void build(const QueryDesc& q, const Smem& sm, const uint32_t* aux, int buf, int wb,
                                               unsigned long long s, unsigned long long e, int hw, int nh) {
    constexpr uint32_t nwords = S::tile_rows / 32;
    constexpr uint32_t per = nwords / 32;
    constexpr int nb = S::n_bitmaps;
    const int lane = threadIdx.x & 31;
    unsigned long long* hcur = helper_cursor(sm);
    cp_async_wait_all();
    __syncwarp();
    static_for<nb>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int c = S::bcol(j);
      constexpr bool is_rle = S::enc(c) == ENC_RLE;
      constexpr bool e64 = S::e64(c);
      if (j % nh != hw) return;
      const ColDesc& cd = q.cols[c];
      uint32_t* B = sm.bm + ((size_t)buf * nb + j) * nwords;
      uint32_t* P = sm.pre + ((size_t)buf * nb + j) * (nwords + 1);
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) B[k * 32 + lane] = 0;
      __syncwarp();
      const unsigned long long cur = hcur[j];
      const uint32_t avail = sm.wcnt[wb * kMaxBitmapCols + j];
      const uint8_t* win = sm.win + ((size_t)wb * nb + j) * kWin * 16;
      unsigned long long cnt = 0;
      int eq = 0;
      for (unsigned long long base = 0;; base += 32) {
        const unsigned long long idx = cur + base + lane;
        long long x = 0;
        bool have = true;
        if (base + lane < avail) {
          if constexpr (e64) x = reinterpret_cast<const long long*>(win)[base + lane];
          else x = reinterpret_cast<const int*>(win)[base + lane];
        } else if (idx < cd.n) {
          x = ldg_val(cd.ends, idx, e64);
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
      // word prefix popcounts: lane owns words [lane * per, lane * per + per)
      uint32_t wv[per];
      uint32_t local = 0;
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        wv[k] = B[lane * per + k];
        local += __popc(wv[k]);
      }
      uint32_t incl = local;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
      }
      uint32_t run = incl - local;
#pragma unroll
      for (uint32_t k = 0; k < per; ++k) {
        P[lane * per + k] = run;
        run += __popc(wv[k]);
      }
      if (lane == 31) P[nwords] = incl;
      if (lane == 0) {
        sm.tcur[buf * kMaxBitmapCols + j] = cur;
        hcur[j] = cur + cnt + (unsigned long long)eq;
      }
      __syncwarp();
    });
    // pass bitmaps: predicates with a pass-bitmap slot (on RLE / index
    // columns), evaluated once per run / listed row
    const uint32_t rows = (uint32_t)(e - s);
    static_for<S::n_preds>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (S::ppbm(i) != 0xFF) {
        constexpr int c = S::pcol(i);
        constexpr int j = S::bslot(c);
        constexpr bool e64 = S::e64(c), v64 = S::v64(c);
        if (j % nh != hw) return;
        const ColDesc& cd = q.cols[c];
        uint32_t* PB = sm.pbm + ((size_t)buf * S::n_pbm + S::ppbm(i)) * nwords;
        const uint32_t nset = sm.pre[((size_t)buf * nb + j) * (nwords + 1) + nwords];
        const unsigned long long cur = sm.tcur[buf * kMaxBitmapCols + j];
        const uint8_t* win = sm.win + ((size_t)wb * nb + j) * kWin * 16;
        const uint32_t avail = sm.wcnt[wb * kMaxBitmapCols + j];
        auto end_at = [&](uint32_t k) -> unsigned long long {
          if (k < avail) {
            if constexpr (e64) return (unsigned long long)reinterpret_cast<const long long*>(win)[k];
            else return (unsigned long long)reinterpret_cast<const int*>(win)[k];
          }
          return (unsigned long long)ldg_val(cd.ends, cur + k, e64);
        };
        auto val_at = [&](uint32_t k) -> long long {
          if (k < avail) {
            const uint8_t* v = win + kWin * 8;
            if constexpr (v64) return reinterpret_cast<const long long*>(v)[k];
            else return (long long)reinterpret_cast<const int*>(v)[k];
          }
          return ldg_val(cd.vals, cur + k, v64);
        };
        if constexpr (S::enc(c) == ENC_RLE) {
#pragma unroll
          for (uint32_t k = 0; k < per; ++k) PB[k * 32 + lane] = 0u;
          __syncwarp();
          // nset boundaries inside the tile: nset + 1 runs, the last one clipped
          for (uint32_t k = lane; k <= nset; k += 32) {
            const uint32_t a = k == 0 ? 0u : (uint32_t)(end_at(k - 1) - s);
            const unsigned long long x = end_at(k);
            const uint32_t b = x - s < rows ? (uint32_t)(x - s) : rows;
            if (fast_pred_value<S, i>(q, aux, val_at(k))) fill_bits(PB, a, b);
          }
        } else {
          const bool base_pass = fast_pred_value<S, i>(q, aux, cd.base);
#pragma unroll
          for (uint32_t k = 0; k < per; ++k) {
            const uint32_t w = k * 32 + lane;
            const uint32_t lo = w * 32;
            uint32_t m = base_pass ? ~0u : 0u;
            if (lo >= rows) m = 0u;
            else if (rows - lo < 32) m &= (1u << (rows - lo)) - 1u;
            PB[w] = m;
          }
          __syncwarp();
          for (uint32_t k = lane; k < nset; k += 32) {
            const uint32_t o = (uint32_t)(end_at(k) - s);
            if (fast_pred_value<S, i>(q, aux, val_at(k)) != base_pass) atomicXor(&PB[o >> 5], 1u << (o & 31));
          }
        }
        __syncwarp();
      }
    });
  }
};

}  // namespace cq
