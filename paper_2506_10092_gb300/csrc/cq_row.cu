// cq_row.cu -- row-mode fused kernel: queries that reference bit-packed,
// dictionary or plain columns (every row is an item), alongside any RLE and
// index columns (aligned through per-tile bitmaps, Section 6 Alignment).
//
// Each CTA (one or two per SM) walks a contiguous range of tiles with a
// software pipeline:
//  * 16, 24 or 28 compute warps filter and aggregate tile t;
//  * one helper warp builds the run-end / position bitmaps (and the pass
//    bitmaps of run-length predicates) of tile t+1 from windows it
//    prefetched with cp.async during tile t-1, and prefetches the windows
//    of tile t+2;
//  * the helper's lane 0 keeps `stages` tiles of the row-level columns in
//    flight with 1-D bulk copies (TMA engine) completing on mbarriers.
// One CTA barrier separates tiles; the group table is flushed to the global
// accumulators when it fills.
#include <cuda_runtime.h>

#include "cq_internal.h"
#include "cq_rowpath.cuh"

namespace cq {

template <int NCW, int GPW, int MINB>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB) row_query_kernel(const __grid_constant__ QueryDesc q) {
  const unsigned long long t_begin = q.tile0 + (unsigned long long)blockIdx.x * q.n_tiles / gridDim.x;
  const unsigned long long t_end = q.tile0 + (unsigned long long)(blockIdx.x + 1) * q.n_tiles / gridDim.x;
  if (t_begin >= t_end) return;
  row_range<NCW, GPW>(q, carve(q), t_begin, t_end);
}


// (compute warps, 32-row groups per warp per tile, CTAs per SM)
#define CQ_ROW_SHAPES(X) \
  X(16, 2, 1) X(16, 4, 1) X(16, 8, 1) X(16, 16, 1) X(16, 2, 2) X(16, 4, 2) X(16, 8, 2) X(16, 16, 2) X(24, 8, 1) X(28, 8, 1)

cudaError_t row_kernel_set_smem(int bytes) {
  cudaError_t e = cudaSuccess;
#define CQ_SET(N, G, M)                                                                                   \
  if (e == cudaSuccess)                                                                                   \
    e = cudaFuncSetAttribute(row_query_kernel<N, G, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  CQ_ROW_SHAPES(CQ_SET)
#undef CQ_SET
  return e;
}

// ncw field: 16 one CTA of 16 compute warps, 8 two such CTAs, 24 / 28 one
// CTA of 24 / 28
void row_shape(const QueryDesc& q, int* ncw, int* gpw, int* minb) {
  *ncw = (q.ncw == 24 || q.ncw == 28) ? q.ncw : 16;
  *gpw = (int)(q.tile_rows / (*ncw * 32));
  *minb = q.ncw == 8 ? 2 : 1;
}

cudaError_t launch_row_kernel(const QueryDesc& q, unsigned grid, cudaStream_t s) {
  int ncw, gpw, minb;
  row_shape(q, &ncw, &gpw, &minb);
  bool launched = false;
#define CQ_GO(N, G, M)                                                                \
  if (!launched && ncw == N && gpw == G && minb == M) {                               \
    row_query_kernel<N, G, M><<<grid, (N + 1) * 32, q.smem_bytes, s>>>(q);            \
    launched = true;                                                                  \
  }
  CQ_ROW_SHAPES(CQ_GO)
#undef CQ_GO
  if (!launched) return cudaErrorInvalidConfiguration;
  return cudaGetLastError();
}

}  // namespace cq
