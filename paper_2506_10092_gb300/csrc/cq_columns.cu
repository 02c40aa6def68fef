// cq_columns.cu -- column validation / statistics kernels, the materialising
// alignment of k RLE columns, and the expansion kernels of the
// decompress-then-scan comparison path.
#include <cuda_runtime.h>

#include <climits>

#include "cq_device.cuh"
#include "cq_internal.h"

namespace cq {

// ------------------------------------------------------------------ column checks
struct CheckOut {
  int err;                 // cq_status of the first violation seen
  int pad;
  long long min_raw, max_raw;
};

__device__ __forceinline__ void block_minmax(long long lmin, long long lmax, CheckOut* out) {
  __shared__ long long smin[32], smax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d; d >>= 1) {
    lmin = min(lmin, __shfl_down_sync(0xFFFFFFFFu, lmin, d));
    lmax = max(lmax, __shfl_down_sync(0xFFFFFFFFu, lmax, d));
  }
  if (lane == 0) {
    smin[warp] = lmin;
    smax[warp] = lmax;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x / 32;
    lmin = lane < nw ? smin[lane] : LLONG_MAX;
    lmax = lane < nw ? smax[lane] : LLONG_MIN;
    for (int d = 16; d; d >>= 1) {
      lmin = min(lmin, __shfl_down_sync(0xFFFFFFFFu, lmin, d));
      lmax = max(lmax, __shfl_down_sync(0xFFFFFFFFu, lmax, d));
    }
    if (lane == 0) {
      atomicMin(&out->min_raw, lmin);
      atomicMax(&out->max_raw, lmax);
    }
  }
}

// RLE: ends strictly increasing, last == n_rows; range of run values.
__global__ void check_rle_kernel(const void* vals, bool v64, const void* ends, bool e64, unsigned long long n,
                                 unsigned long long n_rows, CheckOut* out) {
  long long lmin = LLONG_MAX, lmax = LLONG_MIN;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long x = ldg_val(ends, i, e64);
    const long long prev = i ? ldg_val(ends, i - 1, e64) : 0;
    if (x <= prev) atomicCAS(&out->err, 0, (int)CQ_ERR_UNSORTED);
    if (i == n - 1 && (unsigned long long)x != n_rows) atomicCAS(&out->err, 0, (int)CQ_ERR_SIZE_MISMATCH);
    const long long v = ldg_val(vals, i, v64);
    lmin = min(lmin, v);
    lmax = max(lmax, v);
  }
  block_minmax(lmin, lmax, out);
}

// Index: positions strictly increasing and in [0, n_rows); range of values.
__global__ void check_index_kernel(const void* vals, bool v64, const void* pos, bool p64, unsigned long long n,
                                   unsigned long long n_rows, CheckOut* out) {
  long long lmin = LLONG_MAX, lmax = LLONG_MIN;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long x = ldg_val(pos, i, p64);
    if (i && x <= ldg_val(pos, i - 1, p64)) atomicCAS(&out->err, 0, (int)CQ_ERR_UNSORTED);
    if (x < 0 || (unsigned long long)x >= n_rows) atomicCAS(&out->err, 0, (int)CQ_ERR_INVALID_ARG);
    const long long v = ldg_val(vals, i, v64);
    lmin = min(lmin, v);
    lmax = max(lmax, v);
  }
  block_minmax(lmin, lmax, out);
}

// Packed / dictionary codes: range of the unsigned fields (signed view for
// 64-bit fields); codes must be below n_entries.
// One thread per row: the row's field (codes of a dictionary column must lie
// below its size), folded into the column's min / max.
__global__ void check_packed_kernel(const uint32_t* words, unsigned long long n_words, uint32_t bw,
                                    unsigned long long n_rows, unsigned long long limit, CheckOut* out) {
  long long lmin = LLONG_MAX, lmax = LLONG_MIN;
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < n_rows;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long bit = r * bw;
    const unsigned long long q = bit >> 5;
    const uint32_t sh = (uint32_t)(bit & 31);
    const uint32_t w0 = __ldg(words + q), w1 = q + 1 < n_words ? __ldg(words + q + 1) : 0u;
    uint64_t f = __funnelshift_r(w0, w1, sh);
    if (bw > 32) f |= (uint64_t)__funnelshift_r(w1, q + 2 < n_words ? __ldg(words + q + 2) : 0u, sh) << 32;
    if (bw < 64) f &= (1ull << bw) - 1ull;
    if (limit && f >= limit) atomicCAS(&out->err, 0, (int)CQ_ERR_INVALID_ARG);
    lmin = min(lmin, (long long)f);
    lmax = max(lmax, (long long)f);
  }
  block_minmax(lmin, lmax, out);
}

// Buffers are 16-byte aligned: whole 16-byte vectors first, then the tail.
__global__ void check_plain_kernel(const void* vals, bool v64, unsigned long long n, CheckOut* out) {
  long long lmin = LLONG_MAX, lmax = LLONG_MIN;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long per = v64 ? 2 : 4;
  const unsigned long long nv = n / per;
  const int4* vec = reinterpret_cast<const int4*>(vals);
  for (unsigned long long i = t0; i < nv; i += stride) {
    const int4 x = __ldg(vec + i);
    long long a, b, c, d;
    if (v64) {
      a = (long long)(((unsigned long long)(uint32_t)x.y << 32) | (uint32_t)x.x);
      b = (long long)(((unsigned long long)(uint32_t)x.w << 32) | (uint32_t)x.z);
      c = a;
      d = b;
    } else {
      a = x.x; b = x.y; c = x.z; d = x.w;
    }
    lmin = min(lmin, min(min(a, b), min(c, d)));
    lmax = max(lmax, max(max(a, b), max(c, d)));
  }
  for (unsigned long long i = nv * per + t0; i < n; i += stride) {
    const long long v = ldg_val(vals, i, v64);
    lmin = min(lmin, v);
    lmax = max(lmax, v);
  }
  block_minmax(lmin, lmax, out);
}

cudaError_t run_column_check(const cq_column* c, void* d_out_raw, cudaStream_t s) {
  CheckOut* d_out = reinterpret_cast<CheckOut*>(d_out_raw);
  CheckOut init{0, 0, LLONG_MAX, LLONG_MIN};
  cudaError_t e = cudaMemcpyAsync(d_out, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const unsigned threads = 256;
  auto blocks_for = [](unsigned long long n) {
    unsigned long long b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
  };
  switch (c->enc) {
    case ENC_RLE:
      check_rle_kernel<<<blocks_for(c->n), threads, 0, s>>>(c->vals, c->val_t == CQ_I64, c->ends,
                                                             c->end_t == CQ_I64, c->n, c->n_rows, d_out);
      break;
    case ENC_INDEX:
      check_index_kernel<<<blocks_for(c->n), threads, 0, s>>>(c->vals, c->val_t == CQ_I64, c->ends,
                                                               c->end_t == CQ_I64, c->n, c->n_rows, d_out);
      break;
    case ENC_PACKED:
    case ENC_DICT:
      check_packed_kernel<<<blocks_for(c->n_rows), threads, 0, s>>>(
          reinterpret_cast<const uint32_t*>(c->vals), c->n, c->bit_width, c->n_rows,
          c->enc == ENC_DICT ? (unsigned long long)c->n_entries : 0ull, d_out);
      break;
    case ENC_PLAIN:
      check_plain_kernel<<<blocks_for(c->n_rows), threads, 0, s>>>(c->vals, c->val_t == CQ_I64, c->n_rows, d_out);
      break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ materialising alignment
// One CTA per tile of kAlignTile rows.  The run ends of every column that
// fall in (s, e] are set in per-column bitmaps (bit o <-> end s + o + 1); the
// union gives the segment ends of the tile; the run of column j covering
// the segment that ends at x is the number of column-j ends below x.
constexpr uint32_t kAlignWords = kAlignTile / 32;
constexpr int kAlignThreads = 256;

struct AlignCols {
  const void* ends[kMaxBitmapCols];
  uint8_t e64[kMaxBitmapCols];
  unsigned long long n[kMaxBitmapCols];
  int k;
};

__device__ void align_tile_bits(const AlignCols& A, unsigned long long s, unsigned long long e, uint32_t* bm,
                                uint32_t* pre, uint32_t* ubm, uint32_t* upre, unsigned long long* cur) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < kAlignWords * A.k; i += blockDim.x) bm[i] = 0;
  // cur[2j] = #ends <= s, cur[2j+1] = #ends <= e
  for (int j = warp; j < 2 * A.k; j += kAlignThreads / 32) {
    const int c = j >> 1;
    const unsigned long long key = (j & 1) ? e : s;
    const unsigned long long r = warp_count_below(A.ends[c], A.e64[c], A.n[c], (long long)key, false);
    if (lane == 0) cur[j] = r;
  }
  __syncthreads();
  for (int c = 0; c < A.k; ++c) {
    for (unsigned long long i = cur[2 * c] + threadIdx.x; i < cur[2 * c + 1]; i += blockDim.x) {
      const unsigned long long x = (unsigned long long)ldg_val(A.ends[c], i, A.e64[c]);
      const uint32_t o = (uint32_t)(x - s - 1);
      atomicOr(&bm[c * kAlignWords + (o >> 5)], 1u << (o & 31));
    }
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < kAlignWords; w += blockDim.x) {
    uint32_t u = 0;
    for (int c = 0; c < A.k; ++c) u |= bm[c * kAlignWords + w];
    ubm[w] = u;
  }
  __syncthreads();
  // prefix popcounts: warp c < k for columns, warp k for the union
  for (int c = warp; c <= A.k; c += kAlignThreads / 32) {
    const uint32_t* B = c < A.k ? bm + c * kAlignWords : ubm;
    uint32_t* P = c < A.k ? pre + c * (kAlignWords + 1) : upre;
    const uint32_t per = kAlignWords / 32;
    uint32_t local = 0;
    for (uint32_t t = 0; t < per; ++t) local += __popc(B[lane * per + t]);
    uint32_t incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t run = incl - local;
    for (uint32_t t = 0; t < per; ++t) {
      P[lane * per + t] = run;
      run += __popc(B[lane * per + t]);
    }
    if (lane == 31) P[kAlignWords] = incl;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kAlignThreads) align_count_kernel(AlignCols A, unsigned long long n_rows,
                                                                     unsigned long long* counts) {
  __shared__ uint32_t bm[kMaxBitmapCols * kAlignWords];
  __shared__ uint32_t pre[kMaxBitmapCols * (kAlignWords + 1)];
  __shared__ uint32_t ubm[kAlignWords], upre[kAlignWords + 1];
  __shared__ unsigned long long cur[2 * kMaxBitmapCols];
  const unsigned long long s = blockIdx.x * (unsigned long long)kAlignTile;
  const unsigned long long e = min(s + kAlignTile, n_rows);
  align_tile_bits(A, s, e, bm, pre, ubm, upre, cur);
  if (threadIdx.x == 0) counts[blockIdx.x] = upre[kAlignWords];
}

__global__ void __launch_bounds__(kAlignThreads) align_write_kernel(AlignCols A, unsigned long long n_rows,
                                                                     const unsigned long long* offsets,
                                                                     long long* seg_ends, long long* ridx,
                                                                     unsigned long long capacity) {
  __shared__ uint32_t bm[kMaxBitmapCols * kAlignWords];
  __shared__ uint32_t pre[kMaxBitmapCols * (kAlignWords + 1)];
  __shared__ uint32_t ubm[kAlignWords], upre[kAlignWords + 1];
  __shared__ unsigned long long cur[2 * kMaxBitmapCols];
  const unsigned long long s = blockIdx.x * (unsigned long long)kAlignTile;
  const unsigned long long e = min(s + kAlignTile, n_rows);
  align_tile_bits(A, s, e, bm, pre, ubm, upre, cur);
  for (uint32_t w = threadIdx.x; w < kAlignWords; w += blockDim.x) {
    uint32_t u = ubm[w];
    uint32_t r = upre[w];
    while (u) {
      const int b = __ffs(u) - 1;
      u &= u - 1;
      const uint32_t o = w * 32 + b;
      const unsigned long long idx = offsets[blockIdx.x] + r++;
      if (idx >= capacity) continue;
      seg_ends[idx] = (long long)(s + o + 1);
      for (int c = 0; c < A.k; ++c)
        ridx[(size_t)c * capacity + idx] =
            (long long)(cur[2 * c] + rank_excl(bm + c * kAlignWords, pre + c * (kAlignWords + 1), o));
    }
  }
}

cudaError_t align_segments(cq_column* const* cols, uint32_t k, cudaStream_t s, void* scratch_counts,
                           unsigned long long n_tiles, unsigned long long n_rows, long long* seg_ends,
                           long long* ridx, unsigned long long capacity, unsigned long long* host_counts,
                           unsigned long long* n_segments) {
  AlignCols A{};
  A.k = (int)k;
  for (uint32_t j = 0; j < k; ++j) {
    A.ends[j] = cols[j]->ends;
    A.e64[j] = cols[j]->end_t == CQ_I64;
    A.n[j] = cols[j]->n;
  }
  unsigned long long* d_counts = reinterpret_cast<unsigned long long*>(scratch_counts);
  align_count_kernel<<<(unsigned)n_tiles, kAlignThreads, 0, s>>>(A, n_rows, d_counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(host_counts, d_counts, n_tiles * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  unsigned long long run = 0;
  for (unsigned long long t = 0; t < n_tiles; ++t) {
    const unsigned long long c = host_counts[t];
    host_counts[t] = run;
    run += c;
  }
  *n_segments = run;
  if (run > capacity || capacity == 0) return cudaSuccess;
  e = cudaMemcpyAsync(d_counts, host_counts, n_tiles * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  align_write_kernel<<<(unsigned)n_tiles, kAlignThreads, 0, s>>>(A, n_rows, d_counts, seg_ends, ridx, capacity);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------ decompress-then-scan expansion
// Expand a column to one int64 per row (dictionary: code; packed: base + field).
__global__ void expand_packed_kernel(const uint32_t* words, unsigned long long n_words, uint32_t bw, long long base,
                                     unsigned long long n_rows, long long* out) {
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < n_rows;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long bit = r * bw;
    const unsigned long long q = bit >> 5;
    const uint32_t sh = (uint32_t)(bit & 31);
    const uint32_t w0 = __ldg(words + q), w1 = q + 1 < n_words ? __ldg(words + q + 1) : 0u;
    uint64_t f = __funnelshift_r(w0, w1, sh);
    if (bw > 32) f |= (uint64_t)__funnelshift_r(w1, q + 2 < n_words ? __ldg(words + q + 2) : 0u, sh) << 32;
    if (bw < 64) f &= (1ull << bw) - 1ull;
    out[r] = (long long)(f + (unsigned long long)base);
  }
}

__global__ void expand_plain_kernel(const void* vals, bool v64, unsigned long long n, long long* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    out[i] = ldg_val(vals, i, v64);
}

__global__ void fill_kernel(long long v, unsigned long long n, long long* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    out[i] = v;
}

__global__ void scatter_index_kernel(const void* vals, bool v64, const void* pos, bool p64, unsigned long long n,
                                     long long* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    out[ldg_val(pos, i, p64)] = ldg_val(vals, i, v64);
}

// RLE: one thread per run writes that run's rows.
__global__ void expand_rle_kernel(const void* vals, bool v64, const void* ends, bool e64, unsigned long long n_runs,
                                  long long* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n_runs;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long b = i ? (unsigned long long)ldg_val(ends, i - 1, e64) : 0ull;
    const unsigned long long e = (unsigned long long)ldg_val(ends, i, e64);
    const long long v = ldg_val(vals, i, v64);
    for (unsigned long long r = b; r < e; ++r) out[r] = v;
  }
}

cudaError_t expand_column(const cq_column* c, long long* out, cudaStream_t s, int num_sms) {
  const unsigned grid = (unsigned)(num_sms * 8);
  switch (c->enc) {
    case ENC_RLE:
      expand_rle_kernel<<<grid, 256, 0, s>>>(c->vals, c->val_t == CQ_I64, c->ends, c->end_t == CQ_I64, c->n, out);
      break;
    case ENC_PACKED:
      expand_packed_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(c->vals), c->n, c->bit_width, c->base,
                                                c->n_rows, out);
      break;
    case ENC_DICT:
      expand_packed_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(c->vals), c->n, c->bit_width, 0,
                                                c->n_rows, out);
      break;
    case ENC_INDEX:
      fill_kernel<<<grid, 256, 0, s>>>(c->base, c->n_rows, out);
      scatter_index_kernel<<<grid, 256, 0, s>>>(c->vals, c->val_t == CQ_I64, c->ends, c->end_t == CQ_I64, c->n, out);
      break;
    case ENC_PLAIN:
      expand_plain_kernel<<<grid, 256, 0, s>>>(c->vals, c->val_t == CQ_I64, c->n_rows, out);
      break;
  }
  return cudaGetLastError();
}

}  // namespace cq

namespace cq {

// Launchers of the alignment kernels over raw device run-end arrays, for
// callers that hold no column handles (the allocation-free entry point).
cudaError_t align_launch_count_raw(const void* const* ends, const uint8_t* e64, const unsigned long long* n, uint32_t k,
                                   unsigned long long n_rows, unsigned long long n_tiles, unsigned long long* counts,
                                   cudaStream_t s) {
  AlignCols A{};
  A.k = (int)k;
  for (uint32_t j = 0; j < k; ++j) {
    A.ends[j] = ends[j];
    A.e64[j] = e64[j];
    A.n[j] = n[j];
  }
  align_count_kernel<<<(unsigned)n_tiles, kAlignThreads, 0, s>>>(A, n_rows, counts);
  return cudaGetLastError();
}

cudaError_t align_launch_write_raw(const void* const* ends, const uint8_t* e64, const unsigned long long* n, uint32_t k,
                                   unsigned long long n_rows, unsigned long long n_tiles,
                                   const unsigned long long* offsets, long long* seg_ends, long long* ridx,
                                   unsigned long long capacity, cudaStream_t s) {
  AlignCols A{};
  A.k = (int)k;
  for (uint32_t j = 0; j < k; ++j) {
    A.ends[j] = ends[j];
    A.e64[j] = e64[j];
    A.n[j] = n[j];
  }
  align_write_kernel<<<(unsigned)n_tiles, kAlignThreads, 0, s>>>(A, n_rows, offsets, seg_ends, ridx, capacity);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ bounded-wait self-test
// One thread waits on an mbarrier that nothing will complete, with the
// bounded wait the fused kernels use, and records the status it ends with.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  *status = 0;
  mbar_wait_bounded(&bar, 0, status, limit_ns);
}

cudaError_t launch_bounded_wait_selftest(uint64_t limit_ns, int* status, cudaStream_t s) {
  bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(limit_ns, status);
  return cudaGetLastError();
}

}  // namespace cq
