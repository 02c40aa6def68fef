// cq_batch.cu -- persistent kernel of a query batch.
//
// Many queries, over tables (or partitions) of very different sizes, run in
// one launch.  The host cuts every query's tiles into work items (query, tile
// range), orders them larger first, and uploads them with the queries'
// descriptors.  Each CTA of a one- (or two-) CTA-per-SM grid repeatedly takes the next
// item from a global counter, copies that query's descriptor into shared
// memory, lays out the dynamic shared memory for it, and walks the item's
// tiles with the one-query steps: segment mode (cq_seg.cuh) or row mode with
// its helper warp (cq_rowpath.cuh).  Each item flushes its group table into
// the query's own global accumulators, so items of one query may run on any
// CTAs in any order.  The batch kernel's block is the row-mode shape, 16
// compute warps plus the helper warp; in segment mode the helper warp only
// joins the block barriers.
#include <cuda_runtime.h>

#include "cq_internal.h"
#include "cq_rowpath.cuh"
#include "cq_seg.cuh"

namespace cq {

constexpr int kBatchThreads = (kWarps + 1) * 32;
static_assert(sizeof(QueryDesc) % 8 == 0, "descriptor is copied in 8-byte words");

// MINB CTAs per SM: 1, or 2 when every query of the batch was planned within
// half an SM's shared memory (more resident warps hide more latency).
template <int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB) batch_query_kernel(BatchCtl* ctl) {
  __shared__ __align__(16) QueryDesc qs;
  __shared__ unsigned long long item_id;
  const uint32_t n_items = ctl->n_items;
  for (;;) {
    // the previous item is finished with every shared-memory word; its
    // generic accesses are ordered before the next item's bulk copies
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) item_id = atomicAdd(&ctl->next_item, 1ull);
    __syncthreads();
    const unsigned long long it = item_id;
    if (it >= n_items) break;
    const BatchItem item = ctl->items[it];
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(ctl->descs + item.query);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&qs);
    for (uint32_t i = threadIdx.x; i < sizeof(QueryDesc) / 8; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const Smem sm = carve(qs);
    const unsigned long long t0 = item.t_begin, t1 = item.t_begin + item.n_tiles;
    const uint32_t gpw = qs.tile_rows / (kWarps * 32);
    // batches plan 4096- or 8192-row tiles only: two tile walks per mode keep
    // the kernel's code small enough for the instruction cache
    if (qs.seg_mode) {
      if (gpw == 8) seg_range<8>(qs, sm, t0, t1);
      else seg_range<16>(qs, sm, t0, t1);
    } else {
      if (gpw == 8) row_range<kWarps, 8>(qs, sm, t0, t1);
      else row_range<kWarps, 16>(qs, sm, t0, t1);
    }
  }
}

cudaError_t batch_kernel_static_smem(int minb, size_t* bytes) {
  cudaFuncAttributes a;
  const cudaError_t e = minb == 2 ? cudaFuncGetAttributes(&a, batch_query_kernel<2>)
                                  : cudaFuncGetAttributes(&a, batch_query_kernel<1>);
  if (e == cudaSuccess) *bytes = a.sharedSizeBytes;
  return e;
}

cudaError_t batch_kernel_set_smem(int minb, size_t bytes) {
  return minb == 2
             ? cudaFuncSetAttribute(batch_query_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
             : cudaFuncSetAttribute(batch_query_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_batch_init(const BatchCtl* ctl, cudaStream_t s, unsigned grid);       // cq_query.cu
cudaError_t launch_batch_finalize(const BatchCtl* ctl, cudaStream_t s, unsigned grid);   // cq_query.cu

cudaError_t launch_batch(BatchCtl* ctl_dev, cudaStream_t s, unsigned grid, int minb, size_t dyn_smem,
                         unsigned aux_grid) {
  cudaError_t e = launch_batch_init(ctl_dev, s, aux_grid);
  if (e != cudaSuccess) return e;
  if (minb == 2) batch_query_kernel<2><<<grid, kBatchThreads, dyn_smem, s>>>(ctl_dev);
  else batch_query_kernel<1><<<grid, kBatchThreads, dyn_smem, s>>>(ctl_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_batch_finalize(ctl_dev, s, aux_grid);
}

}  // namespace cq
