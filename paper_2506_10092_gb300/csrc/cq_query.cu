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

#include "cq_phases.cuh"

namespace cq {

size_t query_kernel_smem(const QueryDesc& q) { return smem_layout(q).total; }

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
    const unsigned long long cur = sm.tcur[j];
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

// ------------------------------------------------------------------ segment-mode kernel
// GPW: groups of 32 segments per warp per tile (tile_rows / kThreads).
template <int GPW>
__global__ void __launch_bounds__(kThreads, 1) seg_query_kernel(const __grid_constant__ QueryDesc q) {
  const Smem sm = carve(q);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t T = q.tile_rows;
  const uint32_t nwords = T / 32;
  const unsigned long long t_begin = (unsigned long long)blockIdx.x * q.n_tiles / gridDim.x;
  const unsigned long long t_end = (unsigned long long)(blockIdx.x + 1) * q.n_tiles / gridDim.x;
  if (t_begin >= t_end) return;

  for (uint32_t sl = threadIdx.x; sl < q.table_slots; sl += blockDim.x) reset_slot(q, sm, sl);
  if (threadIdx.x < 8) sm.misc[threadIdx.x] = 0;
  if (threadIdx.x < 2 * kMaxBitmapCols) sm.flags[threadIdx.x] = 0;
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
  tv.stage = nullptr;
  tv.aux = aux_smem ? sm.aux : q.aux;
  tv.nwords = nwords;
  uint32_t rows_since_flush = 0;
  uint16_t* mylist = sm.clist + warp * (GPW * 32);
  const uint32_t wbase = warp * (GPW * 32);

  for (unsigned long long t = t_begin; t < t_end; ++t) {
    const unsigned long long s = t * T;
    const unsigned long long e = (s + T < q.n_rows) ? s + T : q.n_rows;
    const uint32_t rows = (uint32_t)(e - s);
    build_bitmaps(q, sm, s, e, nwords);
    build_segments(q, sm, nwords, rows);
    const uint32_t pm = phase_filter<true, GPW>(q, tv, sm.seg, wbase, (uint32_t)sm.misc[2]);
    const uint32_t n_pass = compact<GPW>(pm, wbase, mylist);
    phase_aggregate<true, 2>(q, sm, tv, sm.seg, mylist, n_pass, s);
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
          if (!fits) report(q, CQ_ERR_OVERFLOW, 3ull + ((unsigned long long)idx << 8), g, x.lo);
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
template <int GPW>
__global__ void row_query_kernel(const __grid_constant__ QueryDesc q);   // cq_row.cu
cudaError_t row_kernel_set_smem(int bytes);
cudaError_t launch_row_kernel(const QueryDesc& q, unsigned grid, cudaStream_t s);

cudaError_t query_kernel_set_smem(size_t bytes) {
  cudaError_t e;
  const int b = (int)bytes;
  if ((e = cudaFuncSetAttribute(seg_query_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(seg_query_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(seg_query_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(seg_query_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  return row_kernel_set_smem(b);
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
  if (!q.seg_mode) return launch_row_kernel(q, grid, s);
  switch (q.tile_rows / kThreads) {
    case 2: seg_query_kernel<2><<<grid, kThreads, q.smem_bytes, s>>>(q); break;
    case 4: seg_query_kernel<4><<<grid, kThreads, q.smem_bytes, s>>>(q); break;
    case 8: seg_query_kernel<8><<<grid, kThreads, q.smem_bytes, s>>>(q); break;
    default: seg_query_kernel<16><<<grid, kThreads, q.smem_bytes, s>>>(q); break;
  }
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
