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
// S provides (all constexpr): tile_rows, n_preds, n_pbm, n_keys, n_aggs,
// one_group, table_dense; per column c: enc, v64, bw, bslot, raw_off,
// stage_off; per predicate i (evaluation order): pcol, pkind, pn32, ppbm;
// per key k: kcol, kremap, kn32; per aggregate i: akind, acol, asw, awide,
// asw32, agw, ared32, aw32, an32, as32, asrc (the first aggregate reading the
// same column value, whose read is reused).
#pragma once

#include "cq_rowpath.cuh"

namespace cq {

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
// Bit g of the result: row wbase + g * GS + lane passes every predicate.
template <class S, uint32_t GS, int GPW>
__device__ __forceinline__ uint32_t fast_filter(const QueryDesc& q, const TileView& t, uint32_t wbase, uint32_t rows) {
  const int lane = threadIdx.x & 31;
  uint32_t valid = 0;
#pragma unroll
  for (int g = 0; g < GPW; ++g) valid |= (wbase + g * GS + lane < rows ? 1u : 0u) << g;
  uint32_t pm = valid;
  static_for<S::n_preds>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int kind = S::pkind(i);
    constexpr int c = S::pcol(i);
    constexpr int E = S::enc(c);
    if constexpr (S::ppbm(i) != 0xFF) {
      // evaluated once per run / listed row by the helper warp: one bit per row
      const uint32_t* PB = t.pbm + (size_t)S::ppbm(i) * (S::tile_rows / 32);
#pragma unroll
      for (int g = 0; g < GPW; ++g) pm &= ((PB[(wbase + g * GS) >> 5] >> lane) & 1u) ? ~0u : ~(1u << g);
    } else if constexpr (kind == PK_FALSE) {
      pm = 0;
    } else if constexpr (kind != PK_TRUE) {
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
          pm &= ok ? ~0u : ~(1u << g);
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
            pm &= ok ? ~0u : ~(1u << g);
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
            pm &= ok ? ~0u : ~(1u << g);
          }
        }
      }
    }
  });
  return pm & valid;
}

// ------------------------------------------------------------------ aggregation
template <class S, int K>
__device__ __forceinline__ bool fast_digit(const QueryDesc& q, const TileView& t, uint32_t o, uint32_t* d,
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
    const unsigned long long dd = (unsigned long long)(v - k.kmin);
    if constexpr (!S::kremap(K)) {
      *d = (uint32_t)dd;
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
// free slot, of group gid's global accumulators).
template <class S, int I>
__device__ __forceinline__ void fast_update(const QueryDesc& q, const Smem& sm, int slot, uint32_t gid, long long v) {
  constexpr int kind = S::akind(I);
  const uint32_t slots = q.table_slots;
  if constexpr (kind == AK_SUM) {
    if (slot >= 0) {
      if constexpr (S::as32(I)) atomicAdd(&sm.tacc32[(size_t)S::asw32(I) * slots + slot], (unsigned)v);
      else if constexpr (!S::awide(I)) smem_add64(&sm.tacc[(size_t)S::asw(I) * slots + slot], v);
      else atomic_add_i128(&sm.tacc[(size_t)S::asw(I) * slots + slot], &sm.tacc[(size_t)(S::asw(I) + 1) * slots + slot],
                           sext(v));
    } else {
      global_add_limbs(gword(q, S::agw(I), gid), gword(q, S::agw(I) + 1, gid), gword(q, S::agw(I) + 2, gid), sext(v));
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
  } else {
    minmax_add(q, sm, a, slot, gid, v, kind == AK_IMIN);
    if (slot >= 0) atomicAdd(slisted(q, sm, a, slot), 1u);
    else atomicAdd(gword(q, a.gw + 1, gid), 1ull);
  }
}

// Aggregate the n_pass compacted rows of this warp, 32 at a time (one per
// lane): group id from the key digits, a shared-table slot, COUNT and every
// aggregate.  A single-group query reduces across the warp first.
template <class S>
__device__ __forceinline__ void fast_aggregate(const QueryDesc& q, const Smem& sm, const TileView& t,
                                               const uint16_t* list, uint32_t n_pass, unsigned long long row0) {
  const int lane = threadIdx.x & 31;
  for (uint32_t j0 = 0; j0 < n_pass; j0 += 32) {
    const uint32_t j = j0 + lane;
    bool act = j < n_pass;
    const uint32_t o = list[act ? j : j0];
    uint32_t gid = 0;
    static_for<S::n_keys>([&](auto K) {
      constexpr int k = decltype(K)::value;
      uint32_t d = 0;
      long long raw = 0;
      if (!fast_digit<S, k>(q, t, o, &d, &raw)) {
        if (act) {
          act = false;
          report(q, CQ_ERR_INVALID_ARG, 1ull + ((unsigned long long)k << 8), row0 + o, (unsigned long long)raw);
        }
        d = 0;
      }
      gid += d * (uint32_t)q.keys[k].stride;
    });
    long long val[S::n_aggs + 1];
    static_for<S::n_aggs>([&](auto A) {
      constexpr int i = decltype(A)::value;
      constexpr int kind = S::akind(i);
      if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX) {
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
            if constexpr (S::as32(i)) atomicAdd(&sm.tacc32[(size_t)S::asw32(i) * q.table_slots], (unsigned)r);
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
        } else if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX) {
          if (act) fast_update<S, i>(q, sm, 0, 0, val[i]);
        } else if constexpr (kind != AK_COUNT) {
          if (act) fast_index_update<S, i>(q, sm, t, 0, 0, o);
        }
      });
    } else {
      int slot = -1;
      if (act) {
        if constexpr (S::table_dense) slot = (int)gid;
        else slot = table_slot(q, sm, gid);
        if (slot >= 0) atomicAdd(scount(q, sm, slot), 1u);
        else atomicAdd(gword(q, 0, gid), 1ull);
      }
      static_for<S::n_aggs>([&](auto A) {
        constexpr int i = decltype(A)::value;
        constexpr int kind = S::akind(i);
        if constexpr (kind == AK_SUM || kind == AK_MIN || kind == AK_MAX) {
          if (act) fast_update<S, i>(q, sm, slot, gid, val[i]);
        } else if constexpr (kind != AK_COUNT) {
          if (act) fast_index_update<S, i>(q, sm, t, slot, gid, o);
        }
      });
    }
  }
}

template <class S>
struct FastBody {
  template <int NCW, int GPW>
  __device__ static __forceinline__ void tile(const QueryDesc& q, const Smem& sm, const TileView& tv, uint32_t wbase,
                                              uint32_t rows, uint16_t* list, unsigned long long row0) {
    constexpr uint32_t GS = NCW * 32;
    const uint32_t pm = fast_filter<S, GS, GPW>(q, tv, wbase, rows);
    const uint32_t n_pass = compact<GPW>(pm, wbase, GS, list);
    fast_aggregate<S>(q, sm, tv, list, n_pass, row0);
  }
};

}  // namespace cq
