// cq_query.cu -- segment-mode fused kernel, global init / finalize kernels
// and the launchers of both fused kernels.
//
// The compressed-domain method (Sections 6-7 of the paper): a table's rows are
// cut into tiles of `tile_rows` rows and each CTA walks a contiguous range of
// tiles.  Alignment (Section 6, Algorithm 1 generalised to k columns): the run
// ends of every RLE column that fall in a tile are set as bits of a tile-long
// bitmap, the listed positions of every index column likewise, and the run
// (or listed entry) covering tile row o is a popcount rank -- the common
// refinement of all runs is never sorted or materialised.  When every
// referenced column is RLE or index-encoded (segment mode, this file) the OR
// of the bitmaps gives the aligned segments themselves and the kernel works
// per segment: SUM adds value x run length, COUNT adds length (Section 7).
// Queries with row-level columns run in the row-mode kernel (cq_row.cu).
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>

#include "cq_internal.h"
#include "cq_seg.cuh"

namespace cq {

size_t query_kernel_smem(const QueryDesc& q) { return smem_layout(q).total; }

// ------------------------------------------------------------------ segment-mode kernel
// GPW: groups of 32 segments per warp per tile (tile_rows / kThreads).  Each
// CTA walks one contiguous range of tiles.
template <int GPW, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) seg_query_kernel(const __grid_constant__ QueryDesc q) {
  const unsigned long long t_begin = q.tile0 + (unsigned long long)blockIdx.x * q.n_tiles / gridDim.x;
  const unsigned long long t_end = q.tile0 + (unsigned long long)(blockIdx.x + 1) * q.n_tiles / gridDim.x;
  if (t_begin >= t_end) return;
  seg_range<GPW>(q, carve(q), t_begin, t_end);
}

// Segment mode walked by runs (run_range): every thread merges the columns'
// boundaries over its share of rows; the block's shared group table is
// flushed once at the end.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) run_query_kernel(const __grid_constant__ QueryDesc q) {
  const Smem sm = carve(q);
  for (uint32_t sl = threadIdx.x; sl < q.table_slots; sl += blockDim.x) reset_slot(q, sm, sl);
  if (threadIdx.x < 8) sm.misc[threadIdx.x] = 0;
  const bool aux_smem = q.aux_words <= kAuxSmemWords;
  if (aux_smem)
    for (uint32_t i = threadIdx.x; i < q.aux_words; i += blockDim.x) sm.aux[i] = __ldg(q.aux + i);
  __syncthreads();
  const unsigned long long r_lo = q.tile0 * q.tile_rows;
  const unsigned long long r_end = (q.tile0 + q.n_tiles) * q.tile_rows;
  run_range(q, sm, aux_smem ? sm.aux : q.aux, r_lo, r_end < q.n_rows ? r_end : q.n_rows);
  __syncthreads();
  flush_table(q, sm);
}

// ------------------------------------------------------------------ init / finalize
// Identity values of group i's global accumulators.
__device__ __forceinline__ void init_group(const QueryDesc& q, size_t i) {
  const size_t G = q.n_groups;
  q.gacc[i] = 0;
  if (q.ghash) q.gkeys[i] = kEmptyGroup;
  for (int ai = 0; ai < q.n_aggs; ++ai) {
    const AggDesc& a = q.aggs[ai];
    switch (a.kind) {
      case AK_SUM:
      case AK_ISUM:
      case AK_SUM2:
      case AK_ISUM2:
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

// Carry the upper halves of a SUM's two 32-bit limb words into the next word
// (w0 + w1 * 2^32 + w2 * 2^64 is unchanged).  Run between the launches of a
// query split by rows, it keeps every word below 2^63 whatever the row count:
// each launch adds fewer than 2^31 limbs (each below 2^32) to a word.
__global__ void fold_sums_kernel(const __grid_constant__ QueryDesc q) {
  const size_t G = q.n_groups;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G; i += (size_t)gridDim.x * blockDim.x) {
    for (int ai = 0; ai < q.n_aggs; ++ai) {
      const AggDesc& a = q.aggs[ai];
      if (a.kind != AK_SUM && a.kind != AK_ISUM && a.kind != AK_SUM2 && a.kind != AK_ISUM2) continue;
      unsigned long long* w0 = &q.gacc[(size_t)a.gw * G + i];
      unsigned long long* w1 = &q.gacc[(size_t)(a.gw + 1) * G + i];
      unsigned long long* w2 = &q.gacc[(size_t)(a.gw + 2) * G + i];
      const unsigned long long c0 = *w0 >> 32;
      *w0 &= 0xFFFFFFFFull;
      const unsigned long long v1 = *w1 + c0;
      *w1 = v1 & 0xFFFFFFFFull;
      *w2 += v1 >> 32;
    }
  }
}

cudaError_t launch_fold_sums(const QueryDesc& q, cudaStream_t s) {
  const unsigned long long nblk = (q.n_groups + 255) / 256;
  const unsigned blocks = (unsigned)(nblk < 4096ull ? nblk : 4096ull);
  fold_sums_kernel<<<blocks ? blocks : 1, 256, 0, s>>>(q);
  return cudaGetLastError();
}

__global__ void init_global_kernel(const __grid_constant__ QueryDesc q) {
  const size_t G = q.n_groups;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G; i += (size_t)gridDim.x * blockDim.x)
    init_group(q, i);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *q.err = 0;
    *q.out_count = 0;
  }
}

constexpr int kFinBlock = 1024;

__device__ __forceinline__ bool group_present(const QueryDesc& q, size_t g) {
  if (q.ghash) return q.gkeys[g] != kEmptyGroup;
  return q.gacc[g] != 0 || (q.n_keys == 0 && g == 0);
}

// Finalize runs in three steps over blocks of kFinBlock dense groups: count
// the present groups of each block, scan the block counts, then write each
// present group's key and aggregates to its compacted result row.
__device__ __forceinline__ void fin_count_block(const QueryDesc& q, unsigned blk) {
  const size_t g = blk * (size_t)kFinBlock + threadIdx.x;
  const bool p = g < q.n_groups && group_present(q, g);
  const int c = __syncthreads_count(p);
  if (threadIdx.x == 0) q.block_counts[blk] = (unsigned)c;
}

__global__ void finalize_count_kernel(const __grid_constant__ QueryDesc q) { fin_count_block(q, blockIdx.x); }

__device__ __forceinline__ void fin_scan(const QueryDesc& q, unsigned n_blocks) {
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

__global__ void finalize_scan_kernel(const __grid_constant__ QueryDesc q, unsigned n_blocks) { fin_scan(q, n_blocks); }

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

// ------------------------------------------------------------------ VAR / STD
// n / d rounded once to the nearest double (ties to even) for a 256-bit n
// (limbs n[0] least significant) and a 128-bit d = (d1, d0) > 0: restoring
// long division, one quotient bit per step, until 64 significant quotient
// bits are known; later quotient bits and the remainder make a sticky bit
// below the double's rounding position.
__device__ double div_rn_256(const unsigned long long n[4], unsigned long long d0, unsigned long long d1) {
  int top_bit = 255;
  while (top_bit >= 0 && !((n[top_bit >> 6] >> (top_bit & 63)) & 1ull)) --top_bit;
  if (top_bit < 0) return 0.0;
  unsigned long long r0 = 0, r1 = 0, r2 = 0;   // remainder, below 2 d < 2^129
  auto step = [&](unsigned long long in) -> bool {
    r2 = (r2 << 1) | (r1 >> 63);
    r1 = (r1 << 1) | (r0 >> 63);
    r0 = (r0 << 1) | in;
    const bool ge = r2 != 0 || r1 > d1 || (r1 == d1 && r0 >= d0);
    if (ge) {
      const unsigned long long b = r0 < d0 ? 1ull : 0ull;
      r0 -= d0;
      r1 = r1 - d1 - b;
      r2 = 0;
    }
    return ge;
  };
  unsigned long long top = 0;
  int got = 0, e = 0;
  bool sticky = false;
  for (int i = top_bit; i >= 0; --i) {
    const bool qb = step((n[i >> 6] >> (i & 63)) & 1ull);
    if (got < 64) {
      if (got || qb) {
        top = (top << 1) | (qb ? 1ull : 0ull);
        ++got;
      }
    } else {
      sticky = sticky || qb;
      ++e;
    }
  }
  while (got < 64) {
    const bool qb = step(0);
    if (got || qb) {
      top = (top << 1) | (qb ? 1ull : 0ull);
      ++got;
    }
    --e;
  }
  sticky = sticky || (r0 | r1 | r2) != 0;
  return scalbn(__ull2double_rn(top | (sticky ? 1ull : 0ull)), e);
}

// Variance of a group (Section 7: from COUNT, SUM and the sum of squares):
// (n * s2 - s1^2) / (n * (n or n - 1)), exact up to the final rounding; 0
// when the denominator is 0.  s2 >= 0 below 2^126, |s1| below 2^127.
__device__ double variance(unsigned long long n, I128 s1, I128 s2, bool sample) {
  const unsigned long long den1 = sample ? n - 1 : n;
  if (n == 0 || den1 == 0) return 0.0;
  // |s1|
  unsigned long long a0 = s1.lo, a1 = (unsigned long long)s1.hi;
  if (s1.hi < 0) {
    a0 = ~a0 + 1ull;
    a1 = ~a1 + (a0 == 0 ? 1ull : 0ull);
  }
  // s1^2 (256 bits): a0^2 + 2 a0 a1 2^64 + a1^2 2^128
  unsigned long long sq[4];
  {
    const unsigned long long p00l = a0 * a0, p00h = __umul64hi(a0, a0);
    const unsigned long long p01l = a0 * a1, p01h = __umul64hi(a0, a1);
    const unsigned long long p11l = a1 * a1, p11h = __umul64hi(a1, a1);
    // cross term doubled: (p01h:p01l) * 2 -> 129 bits
    const unsigned long long c2 = p01h >> 63, x1 = (p01h << 1) | (p01l >> 63), x0 = p01l << 1;
    sq[0] = p00l;
    unsigned long long t = p00h + x0;
    unsigned long long c = t < p00h ? 1ull : 0ull;
    sq[1] = t;
    t = p11l + x1;
    unsigned long long cc = t < p11l ? 1ull : 0ull;
    const unsigned long long t2 = t + c;
    cc += t2 < t ? 1ull : 0ull;
    sq[2] = t2;
    sq[3] = p11h + c2 + cc;
  }
  // n * s2 (s2 < 2^126: at most 190 bits)
  unsigned long long ns[4];
  {
    const unsigned long long s0 = s2.lo, s1w = (unsigned long long)s2.hi;
    const unsigned long long l0 = n * s0, h0 = __umul64hi(n, s0);
    const unsigned long long l1 = n * s1w, h1 = __umul64hi(n, s1w);
    ns[0] = l0;
    ns[1] = h0 + l1;
    ns[2] = h1 + (ns[1] < h0 ? 1ull : 0ull);
    ns[3] = 0;
  }
  // numerator = n s2 - s1^2 >= 0
  unsigned long long num[4];
  unsigned long long borrow = 0;
  for (int i = 0; i < 4; ++i) {
    const unsigned long long x = ns[i], y = sq[i];
    const unsigned long long d = x - y - borrow;
    borrow = (x < y || (x == y && borrow)) ? 1ull : 0ull;
    num[i] = d;
  }
  // denominator n * den1 (128 bits)
  const unsigned long long d0 = n * den1, d1 = __umul64hi(n, den1);
  return div_rn_256(num, d0, d1);
}

// Result row `row` of the group with packed key `key` whose accumulators sit
// at index g (dense domains: key == g).
__device__ __forceinline__ void write_group(const QueryDesc& q, size_t row, unsigned long long key, size_t g) {
  const unsigned long long cnt = q.gacc[g];
  for (uint32_t oc = 0; oc < q.n_out; ++oc) {
    const uint32_t idx = q.out_index[oc];
    if (q.out_is_key[oc]) {
      const KeyDesc& k = q.keys[idx];
      const unsigned long long digit = (key / k.stride) % k.card;
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
          if (!fits) report(q, CQ_ERR_OVERFLOW, 3ull + ((unsigned long long)idx << 8), g, x.lo);
          reinterpret_cast<long long*>(q.out[oc])[row] = (long long)x.lo;
        }
        break;
      }
      case AK_SUM2:
      case AK_ISUM2: {
        // VAR / STD of the shifted values (raw offsets, or value - default):
        // a variance does not change under a shift
        const I128 s1 = read_sum(q, q.aggs[a.pair].gw, g), s2 = read_sum(q, a.gw, g);
        const bool sample = a.op == CQ_VAR_SAMP || a.op == CQ_STD_SAMP;
        const double v = variance(cnt, s1, s2, sample);
        reinterpret_cast<double*>(q.out[oc])[row] = (a.op == CQ_STD_POP || a.op == CQ_STD_SAMP) ? sqrt(v) : v;
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


__device__ __forceinline__ void fin_write_block(const QueryDesc& q, unsigned blk) {
  __shared__ unsigned warp_cnt[kFinBlock / 32];
  const size_t g = blk * (size_t)kFinBlock + threadIdx.x;
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
  const size_t row = q.block_counts[blk] + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
  write_group(q, row, g, g);
}

__global__ void finalize_write_kernel(const __grid_constant__ QueryDesc q) { fin_write_block(q, blockIdx.x); }

// ------------------------------------------------------------------ hash-domain finalize
// Groups of a hash domain sit in the slots of an open-addressing table, in no
// order.  Finalize compacts the occupied slots into (packed key, slot) pairs,
// sorts them by key with a stable least-significant-digit radix sort (8-bit
// digits, as many passes as the packed key has bytes; the packed key orders
// like the key tuple), then writes row r from the r-th pair.

// (key, slot) of the occupied slots of block blk at their compacted rows.
__global__ void __launch_bounds__(kFinBlock) hfin_compact_kernel(const __grid_constant__ QueryDesc q) {
  __shared__ unsigned warp_cnt[kFinBlock / 32];
  const size_t g = blockIdx.x * (size_t)kFinBlock + threadIdx.x;
  const bool p = g < q.n_groups && q.gkeys[g] != kEmptyGroup;
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
  q.skeys[0][row] = q.gkeys[g];
  q.svals[0][row] = (uint32_t)g;
}

constexpr int kSortThreads = 256;   // one element per thread per tile; 8 warps

// Elements [b0, b1) of sort block b out of n (tiles of kSortThreads).
__device__ __forceinline__ void sort_chunk(uint32_t n, uint32_t* b0, uint32_t* b1) {
  const uint32_t nb = gridDim.x;
  const uint32_t chunk = ((n + nb - 1) / nb + kSortThreads - 1) / kSortThreads * kSortThreads;
  const unsigned long long lo = (unsigned long long)blockIdx.x * chunk;
  *b0 = lo < n ? (uint32_t)lo : n;
  *b1 = lo + chunk < n ? (uint32_t)(lo + chunk) : n;
}

// Digit counts of this block's chunk: shist[digit * blocks + block].
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const __grid_constant__ QueryDesc q, int pass) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t n = (uint32_t)*q.out_count;
  uint32_t b0, b1;
  sort_chunk(n, &b0, &b1);
  const unsigned long long* k = q.skeys[pass & 1];
  for (uint32_t i = b0 + threadIdx.x; i < b1; i += kSortThreads) atomicAdd(&h[(k[i] >> (8 * pass)) & 255u], 1u);
  __syncthreads();
  q.shist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a[0, n) in place (one block).
__global__ void __launch_bounds__(1024) scan_u32_kernel(uint32_t* a, uint32_t n) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < n ? a[i] : 0u;
    uint32_t incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t x = lane < (int)(blockDim.x / 32) ? warp_tot[lane] : 0u;
      uint32_t wi = x;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
        if (lane >= d) wi += y;
      }
      warp_tot[lane] = wi - x;
    }
    __syncthreads();
    const uint32_t c0 = carry;
    if (i < n) a[i] = c0 + warp_tot[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_tot[warp] + incl;
    __syncthreads();
  }
}

// Stable scatter of this block's chunk by digit `pass`: tiles in order,
// warps of a tile in order, lanes of a warp in order.
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const __grid_constant__ QueryDesc q, int pass) {
  constexpr int kW = kSortThreads / 32;
  __shared__ uint32_t base[256];
  __shared__ uint32_t tile_tot[256];
  __shared__ uint32_t wcnt[kW][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n = (uint32_t)*q.out_count;
  uint32_t b0, b1;
  sort_chunk(n, &b0, &b1);
  const unsigned long long* kin = q.skeys[pass & 1];
  const uint32_t* vin = q.svals[pass & 1];
  unsigned long long* kout = q.skeys[(pass & 1) ^ 1];
  uint32_t* vout = q.svals[(pass & 1) ^ 1];
  base[threadIdx.x] = q.shist[threadIdx.x * gridDim.x + blockIdx.x];
  for (uint32_t i0 = b0; i0 < b1; i0 += kSortThreads) {
    for (int w = 0; w < kW; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t i = i0 + threadIdx.x;
    const bool valid = i < b1;
    const unsigned long long key = valid ? kin[i] : 0ull;
    const uint32_t val = valid ? vin[i] : 0u;
    const uint32_t d = valid ? (uint32_t)((key >> (8 * pass)) & 255u) : 256u + (uint32_t)lane;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
      for (int w = 0; w < kW; ++w) {
        const uint32_t c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += c;
      }
      tile_tot[threadIdx.x] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base[d] + wcnt[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    base[threadIdx.x] += tile_tot[threadIdx.x];
    __syncthreads();
  }
}

// Row r from the r-th sorted pair (grid-stride).
__global__ void hfin_write_kernel(const __grid_constant__ QueryDesc q, int buf) {
  const unsigned long long n = *q.out_count;
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < n;
       r += (unsigned long long)gridDim.x * blockDim.x)
    write_group(q, (size_t)r, q.skeys[buf][r], (size_t)q.svals[buf][r]);
}

// ------------------------------------------------------------------ batched init / finalize
// The same steps over every query of a batch: blocks of all queries are
// numbered consecutively (init_first / fin_first give each query's first
// block) and a fixed grid strides over them, so one launch configuration
// serves any batch.

// Query owning block b: the last query whose first block is <= b.
__device__ __forceinline__ uint32_t owner_query(const uint32_t* first, uint32_t n_queries, uint32_t b) {
  uint32_t lo = 0, hi = n_queries;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (first[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void batch_init_kernel(const BatchCtl* ctl) {
  const uint32_t nq = ctl->n_queries, nblk = ctl->n_init_blocks;
  for (uint32_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const uint32_t qi = owner_query(ctl->init_first, nq, b);
    const QueryDesc& q = ctl->descs[qi];
    const size_t g0 = (size_t)(b - ctl->init_first[qi]) * kInitGroups;
    const size_t g1 = g0 + kInitGroups < q.n_groups ? g0 + kInitGroups : q.n_groups;
    for (size_t i = g0 + threadIdx.x; i < g1; i += blockDim.x) init_group(q, i);
    if (g0 == 0 && threadIdx.x == 0) {
      *q.err = 0;
      *q.out_count = 0;
    }
  }
}

__global__ void __launch_bounds__(kFinBlock) batch_fin_count_kernel(const BatchCtl* ctl) {
  const uint32_t nq = ctl->n_queries, nblk = ctl->n_fin_blocks;
  for (uint32_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const uint32_t qi = owner_query(ctl->fin_first, nq, b);
    fin_count_block(ctl->descs[qi], b - ctl->fin_first[qi]);
  }
}

__global__ void __launch_bounds__(kFinBlock) batch_fin_scan_kernel(const BatchCtl* ctl) {
  for (uint32_t qi = blockIdx.x; qi < ctl->n_queries; qi += gridDim.x) {
    fin_scan(ctl->descs[qi], ctl->fin_first[qi + 1] - ctl->fin_first[qi]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFinBlock) batch_fin_write_kernel(const BatchCtl* ctl) {
  const uint32_t nq = ctl->n_queries, nblk = ctl->n_fin_blocks;
  for (uint32_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const uint32_t qi = owner_query(ctl->fin_first, nq, b);
    fin_write_block(ctl->descs[qi], b - ctl->fin_first[qi]);
    __syncthreads();   // the block's warp counts are reused by the next block
  }
}

cudaError_t launch_batch_init(const BatchCtl* ctl, cudaStream_t s, unsigned grid) {
  batch_init_kernel<<<grid, 256, 0, s>>>(ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchCtl* ctl, cudaStream_t s, unsigned grid) {
  batch_fin_count_kernel<<<grid, kFinBlock, 0, s>>>(ctl);
  batch_fin_scan_kernel<<<grid, kFinBlock, 0, s>>>(ctl);
  batch_fin_write_kernel<<<grid, kFinBlock, 0, s>>>(ctl);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
template <int GPW>
__global__ void row_query_kernel(const __grid_constant__ QueryDesc q);   // cq_row.cu
cudaError_t row_kernel_set_smem(int bytes);
cudaError_t launch_row_kernel(const QueryDesc& q, unsigned grid, cudaStream_t s);

cudaError_t query_kernel_set_smem(size_t bytes) {
  cudaError_t e;
  const int b = (int)bytes;
  if ((e = cudaFuncSetAttribute(run_query_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(run_query_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
#define CQ_SEG_SET(G, M)                                                                                  \
  if ((e = cudaFuncSetAttribute(seg_query_kernel<G, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  CQ_SEG_SET(2, 1) CQ_SEG_SET(4, 1) CQ_SEG_SET(8, 1) CQ_SEG_SET(16, 1)
  CQ_SEG_SET(2, 2) CQ_SEG_SET(4, 2) CQ_SEG_SET(8, 2) CQ_SEG_SET(16, 2)
  CQ_SEG_SET(2, 3) CQ_SEG_SET(4, 3) CQ_SEG_SET(8, 3) CQ_SEG_SET(16, 3)
#undef CQ_SEG_SET
  return row_kernel_set_smem(b);
}

cudaError_t launch_init_global(const QueryDesc& q, cudaStream_t s) {
  const unsigned long long nblk = (q.n_groups + 255) / 256;
  const unsigned blocks = (unsigned)(nblk < 4096ull ? nblk : 4096ull);
  init_global_kernel<<<blocks ? blocks : 1, 256, 0, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_query(const QueryDesc& q, cudaStream_t s, int num_sms, int ctas_per_sm, uint32_t grid_ctas,
                         const void* row_fn) {
  const unsigned long long want =
      grid_ctas ? (unsigned long long)grid_ctas : (unsigned long long)num_sms * (unsigned long long)ctas_per_sm;
  const unsigned grid = (unsigned)(q.n_tiles < want ? q.n_tiles : want);
  if (grid == 0) return cudaSuccess;
  if (!q.seg_mode) {
    if (!row_fn) return launch_row_kernel(q, grid, s);
    int ncw, gpw, minb;
    row_shape(q, &ncw, &gpw, &minb);
    return launch_row_jit(row_fn, q, grid, ncw, s);
  }
  if (q.run_walk) {
    // every thread of a full grid (at most two CTAs per SM resident) takes a
    // share of the runs
    const unsigned g = grid_ctas ? grid_ctas : (unsigned)num_sms * (unsigned)(ctas_per_sm < 2 ? ctas_per_sm : 2);
    if (ctas_per_sm >= 2) run_query_kernel<2><<<g, kThreads, q.smem_bytes, s>>>(q);
    else run_query_kernel<1><<<g, kThreads, q.smem_bytes, s>>>(q);
    return cudaGetLastError();
  }
  switch (q.tile_rows / kThreads) {
    // two or three CTAs per SM overlap one CTA's barrier-separated phases with
    // the others'
#define CQ_SEG_GO(G)                                                                      \
  case G:                                                                                 \
    if (ctas_per_sm == 3) seg_query_kernel<G, 3><<<grid, kThreads, q.smem_bytes, s>>>(q); \
    else if (ctas_per_sm == 2) seg_query_kernel<G, 2><<<grid, kThreads, q.smem_bytes, s>>>(q); \
    else seg_query_kernel<G, 1><<<grid, kThreads, q.smem_bytes, s>>>(q);                  \
    break;
    CQ_SEG_GO(2) CQ_SEG_GO(4) CQ_SEG_GO(8)
#undef CQ_SEG_GO
    default:
      if (ctas_per_sm == 3) seg_query_kernel<16, 3><<<grid, kThreads, q.smem_bytes, s>>>(q);
      else if (ctas_per_sm == 2) seg_query_kernel<16, 2><<<grid, kThreads, q.smem_bytes, s>>>(q);
      else seg_query_kernel<16, 1><<<grid, kThreads, q.smem_bytes, s>>>(q);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize(const QueryDesc& q, cudaStream_t s) {
  const unsigned nb = (unsigned)((q.n_groups + kFinBlock - 1) / kFinBlock);
  finalize_count_kernel<<<nb, kFinBlock, 0, s>>>(q);
  finalize_scan_kernel<<<1, 1024, 0, s>>>(q, nb);
  if (!q.ghash) {
    finalize_write_kernel<<<nb, kFinBlock, 0, s>>>(q);
    return cudaGetLastError();
  }
  hfin_compact_kernel<<<nb, kFinBlock, 0, s>>>(q);
  const int passes = (q.key_bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    sort_hist_kernel<<<q.sort_blocks, kSortThreads, 0, s>>>(q, p);
    scan_u32_kernel<<<1, 1024, 0, s>>>(q.shist, 256u * q.sort_blocks);
    sort_scatter_kernel<<<q.sort_blocks, kSortThreads, 0, s>>>(q, p);
  }
  hfin_write_kernel<<<q.sort_blocks, 256, 0, s>>>(q, passes & 1);
  return cudaGetLastError();
}

}  // namespace cq
