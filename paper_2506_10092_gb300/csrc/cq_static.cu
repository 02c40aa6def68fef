// cq_static.cu -- the allocation-free form of the materialising alignment.
//
// Some callers cannot allocate device memory on the fly: code that runs under
// a memory budget enforced by someone else (a pre-sized arena, an embedding
// host that owns every allocation), or code that must not call into the CUDA
// allocator at all while it runs.  cq_align_segments_static gives them the
// same result as cq_align_segments without any device allocation: its only
// scratch -- per-tile segment counts and their prefix sums, plus a few status
// words -- lives in one file-scope device array of fixed size that every GPU
// loading this library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "cq_device.cuh"
#include "cq_internal.h"

namespace cq {

constexpr unsigned long long kStaticTiles = CQ_STATIC_ALIGN_MAX_TILES;
constexpr unsigned long long kStaticTileRows = kAlignTile;   // rows per tile of the alignment kernels
static_assert(kStaticTileRows == 4096, "the header states the row limit as CQ_STATIC_ALIGN_MAX_TILES * 4096");

// [0, kStaticTiles): per-tile counts, then their exclusive prefix sums;
// [kStaticTiles]: total segments; [kStaticTiles + 1]: input status (0 ok)
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticTiles + 8];

cudaError_t align_launch_count_raw(const void* const* ends, const uint8_t* e64, const unsigned long long* n, uint32_t k,
                                   unsigned long long n_rows, unsigned long long n_tiles, unsigned long long* counts,
                                   cudaStream_t s);
cudaError_t align_launch_write_raw(const void* const* ends, const uint8_t* e64, const unsigned long long* n, uint32_t k,
                                   unsigned long long n_rows, unsigned long long n_tiles,
                                   const unsigned long long* offsets, long long* seg_ends, long long* ridx,
                                   unsigned long long capacity, cudaStream_t s);

// Run ends must be strictly increasing with the last equal to n_rows (the
// kernels rely on it to stay inside their tiles); violations set the status.
__global__ void static_check_ends_kernel(const void* ends, bool e64, unsigned long long n, unsigned long long n_rows,
                                         unsigned long long* status) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long x = ldg_val(ends, i, e64);
    const long long prev = i ? ldg_val(ends, i - 1, e64) : 0;
    if (x <= prev) atomicCAS(status, 0ull, (unsigned long long)(-(long long)CQ_ERR_UNSORTED));
    if (i == n - 1 && (unsigned long long)x != n_rows)
      atomicCAS(status, 0ull, (unsigned long long)(-(long long)CQ_ERR_SIZE_MISMATCH));
  }
}

// In-place exclusive scan of the per-tile counts by one block; the total
// goes to counts[kStaticTiles].
__global__ void static_scan_kernel(unsigned long long* counts, unsigned long long n_tiles) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned long long base = 0; base < n_tiles; base += blockDim.x) {
    const unsigned long long i = base + threadIdx.x;
    const unsigned long long v = i < n_tiles ? counts[i] : 0ull;
    unsigned long long incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long x = lane < (int)(blockDim.x / 32) ? warp_tot[lane] : 0ull;
      unsigned long long wi = x;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
        if (lane >= d) wi += y;
      }
      warp_tot[lane] = wi - x;
    }
    __syncthreads();
    const unsigned long long c0 = carry;
    if (i < n_tiles) counts[i] = c0 + warp_tot[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_tot[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[kStaticTiles] = carry;
}

// The CUDA context current on this thread (driver entry point looked up
// through the runtime, so the library needs no link against the driver).
static void* current_context() {
  typedef int (*GetCurrent)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<GetCurrent>(f);
  }();
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}

// Device address of the static scratch: looked up (with the device current)
// at the first call in each device context and cached for that context, so a
// context torn down and created again (cudaDeviceReset) gets its own lookup.
static int static_scratch(int device, unsigned long long** out) {
  struct Entry {
    int device;
    void* context;
    unsigned long long* addr;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  void* context = current_context();
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.device == device && e.context == context && context) {
      *out = e.addr;
      return CQ_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess)
    return set_error(CQ_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
  *out = reinterpret_cast<unsigned long long*>(p);
  // a context created after cudaDeviceReset may reuse the old handle value:
  // the entry for this device is replaced, never kept beside it
  for (Entry& x : cache)
    if (x.device == device) {
      x.context = context;
      x.addr = *out;
      return CQ_OK;
    }
  cache.push_back({device, context, *out});
  return CQ_OK;
}

}  // namespace cq

using namespace cq;

extern "C" int cq_align_segments_static(uint32_t k, const void* const* run_ends, const uint32_t* end_is_i64,
                                        const uint64_t* n_runs, uint64_t n_rows, void* cuda_stream,
                                        int64_t* seg_ends, int64_t* ridx, uint64_t capacity,
                                        uint64_t* n_segments) {
  clear_error();
  if (!run_ends || !end_is_i64 || !n_runs || !n_segments) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  if (k == 0 || k > (uint32_t)kMaxBitmapCols) return set_error(CQ_ERR_INVALID_ARG, "k must be in 1..%d", kMaxBitmapCols);
  if (capacity && (!seg_ends || !ridx)) return set_error(CQ_ERR_INVALID_ARG, "NULL output buffer");
  // compared before the tile count is formed, which would wrap near 2^64
  if (n_rows > kStaticTiles * kStaticTileRows)
    return set_error(CQ_ERR_INVALID_ARG,
                     "%llu rows exceed the static alignment limit of %llu rows (%llu tiles of %llu rows)",
                     (unsigned long long)n_rows, kStaticTiles * kStaticTileRows, kStaticTiles, kStaticTileRows);
  const unsigned long long n_tiles = n_rows / kStaticTileRows + (n_rows % kStaticTileRows != 0 ? 1 : 0);
  uint8_t e64[kMaxBitmapCols];
  unsigned long long n[kMaxBitmapCols];
  for (uint32_t j = 0; j < k; ++j) {
    if (n_rows && (!run_ends[j] || n_runs[j] == 0)) return set_error(CQ_ERR_SIZE_MISMATCH, "column %u has no runs", j);
    if (!n_rows && n_runs[j]) return set_error(CQ_ERR_SIZE_MISMATCH, "runs given for an empty column");
    e64[j] = end_is_i64[j] ? 1 : 0;
    n[j] = n_runs[j];
  }
  *n_segments = 0;
  if (n_tiles == 0) return CQ_OK;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  unsigned long long* scratch = nullptr;
  int rc = static_scratch(device, &scratch);
  if (rc != CQ_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned long long* status = scratch + kStaticTiles + 1;
  // the array keeps the previous call's contents: clear the status word
  e = cudaMemsetAsync(status, 0, sizeof(unsigned long long), s);
  for (uint32_t j = 0; j < k && e == cudaSuccess; ++j) {
    static_check_ends_kernel<<<(unsigned)((n[j] + 255) / 256 < 1024 ? (n[j] + 255) / 256 : 1024), 256, 0, s>>>(
        run_ends[j], e64[j], n[j], n_rows, status);
    e = cudaGetLastError();
  }
  unsigned long long st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "run-end check failed: %s", cudaGetErrorString(e));
  if (st) return set_error(-(int)(long long)st, "run ends must be strictly increasing and end at n_rows");
  // every tile's count is overwritten before it is read
  e = align_launch_count_raw(run_ends, e64, n, k, n_rows, n_tiles, scratch, s);
  if (e == cudaSuccess) {
    static_scan_kernel<<<1, 1024, 0, s>>>(scratch, n_tiles);
    e = cudaGetLastError();
  }
  unsigned long long total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, scratch + kStaticTiles, sizeof(total), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "alignment failed: %s", cudaGetErrorString(e));
  *n_segments = total;
  if (total > capacity) return set_error(CQ_ERR_SIZE_MISMATCH, "%llu segments, capacity %llu", total, (unsigned long long)capacity);
  e = align_launch_write_raw(run_ends, e64, n, k, n_rows, n_tiles, scratch, reinterpret_cast<long long*>(seg_ends),
                             reinterpret_cast<long long*>(ridx), capacity, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "alignment failed: %s", cudaGetErrorString(e));
  return CQ_OK;
}
