// cq_internal.h -- internal structures of the cq library (host planner and
// device kernels).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/cq.h"
#include "cq_desc.h"

namespace cq {

// Rows per CTA tile of the materialising alignment kernels (cq_columns.cu);
// the allocation-free entry point (cq_static.cu) sizes its scratch by it.
constexpr uint32_t kAlignTile = 4096;

// ---------------------------------------------------------------- host objects
struct ColumnStats {
  int64_t min_raw = 0, max_raw = -1;     // raw value range (empty when max < min)
  int64_t min_val = 0, max_val = -1;     // logical value range
  uint64_t max_abs_val = 0;              // max |logical value| (saturating)
};

// A planned query: descriptor, aux tables and output description.
struct Planned {
  QueryDesc q;
  std::vector<uint32_t> aux;
  std::vector<uint32_t> out_kind;
  std::vector<int> out_key_col;
  int ctas_per_sm = 1;
  uint32_t grid_ctas = 0;
  bool generic = false;          // row mode: use the generic kernel, not a shape-specialised one
  const void* row_fn = nullptr;  // row mode: the shape-specialised kernel (cq_jit.cu) once resolved
};

// Byte offsets of one query's device buffers inside one allocation.
struct QueryBlock {
  uint64_t gacc, out, hkeys, hsort, aux, err, cnt, blk, total;
};

struct BatchGraph;   // cq_serve.cu
struct TunedShape {  // autotuner choice for a batch signature
  uint64_t key;
  uint32_t tile_rows;
  uint32_t items_per_cta;
};

}  // namespace cq

struct cq_ctx {
  std::atomic<int> refs{1};  // the creator's reference plus one per live column
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  int num_sms = 0;
  size_t smem_optin = 0;     // max dynamic shared memory of one CTA
  size_t smem_two = 0;       // max dynamic shared memory per CTA with two CTAs per SM
  size_t smem_three = 0;     // ... with three CTAs per SM (segment mode)
  std::mutex mu;
  // batches: cached launch graphs and autotuned shapes
  std::mutex batch_mu;
  std::vector<cq::BatchGraph*> graphs;   // owned; freed by the destructor (cq_serve.cu)
  std::vector<cq::TunedShape> tuned;
  size_t batch_smem = 0;     // dynamic shared memory of the batch kernel (one CTA per SM)
  size_t batch_smem_two = 0; // ... and with two CTAs per SM
  ~cq_ctx();
};

struct cq_column {
  cq_ctx* ctx = nullptr;
  std::atomic<int> refs{1};
  uint8_t enc = 0;
  uint64_t n_rows = 0;
  bool owned = false;        // device buffers allocated by the library
  cq_dtype val_t = CQ_I64, end_t = CQ_I64;
  void* vals = nullptr;      // device
  void* ends = nullptr;      // device
  uint64_t n = 0;            // runs / nnz / words / rows
  uint32_t bit_width = 0;
  int64_t base = 0;          // packed base / index default
  cq_dtype logical_t = CQ_I64;
  // dictionary (host)
  std::vector<char> dict_bytes;
  std::vector<uint64_t> dict_offsets;
  uint32_t n_entries = 0;
  cq::ColumnStats stats;
  uint64_t device_bytes = 0;
  ~cq_column();              // drops the column's reference to its context
};

struct cq_table {
  cq_ctx* ctx = nullptr;
  std::vector<cq_column*> cols;
  uint64_t n_rows = 0;
};

struct cq_result {
  cq_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;   // around the fused kernel
  void* dev_block = nullptr;       // one pool allocation holding every device buffer
  size_t dev_bytes = 0;
  cq::QueryDesc desc;              // as launched
  uint32_t n_out = 0;
  std::vector<uint32_t> out_kind;  // 0 int64, 1 uint64, 2 double
  std::vector<int> out_key_col;    // table column of a key output, -1 for aggregates
  std::vector<cq_column*> key_cols;
  int* err_dev = nullptr;
  unsigned long long* count_dev = nullptr;
  bool waited = false;
  int status = CQ_OK;
  uint64_t n_groups = 0;
  std::vector<void*> out_dev;
  std::vector<void*> extra_dev;     // further pool allocations (flat columns of the comparison path)
  std::vector<cq_column*> held_cols; // columns referenced until the result is destroyed
  std::shared_ptr<void> batch_keepalive;  // batch launches: shared device block and events
  bool own_events = true;          // false: the events belong to the batch
  std::unique_ptr<cq::Planned> retry;  // hash-domain queries: the plan, relaunched when its table fills
  uint32_t retries = 0;
};

namespace cq {

// Drop one reference to the context; the last one tears it down.
void ctx_release(cq_ctx* ctx);

// Clear a non-sticky error left by an earlier runtime call, so that the
// error read after a launch belongs to that launch (CQ_DEBUG=1 reports it).
void clear_stale_error(const char* where);

// error reporting (thread-local message)
int set_error(int status, const char* fmt, ...);
void clear_error();

#define CQ_CUDA(call)                                                                           \
  do {                                                                                          \
    cudaError_t _e = (call);                                                                    \
    if (_e != cudaSuccess)                                                                      \
      return set_error(_e == cudaErrorMemoryAllocation ? CQ_ERR_OOM : CQ_ERR_CUDA, "%s failed: %s", \
                       #call, cudaGetErrorString(_e));                                          \
  } while (0)

// Stream-ordered allocation from a context's pool.  Host-side fault
// injection for tests: with CQ_FAULT_INJECT=alloc:N in the environment the
// N-th call of the process (counting from 1) fails with
// cudaErrorMemoryAllocation without calling CUDA.
cudaError_t pool_alloc(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s);

// N when the environment holds CQ_FAULT_INJECT=<kind>:N, else 0 (host-side
// fault injection for tests; kinds "alloc" and "event").
long long fault_inject_at(const char* kind);

// kernels / launchers (cq_query.cu)
cudaError_t launch_query(const QueryDesc& q, cudaStream_t s, int num_sms, int ctas_per_sm, uint32_t grid_ctas,
                         const void* row_fn = nullptr);

// shape-specialised row kernels compiled at run time (cq_jit.cu)
bool jit_enabled();
int jit_row_kernel(const QueryDesc& q, int ncw, int gpw, int minb, int device, size_t smem_limit, const void** fn);
cudaError_t launch_row_jit(const void* fn, const QueryDesc& q, unsigned grid, int ncw, cudaStream_t s);
// compute warps, groups per warp and CTAs per SM of a row-mode descriptor
void row_shape(const QueryDesc& q, int* ncw, int* gpw, int* minb);
cudaError_t launch_init_global(const QueryDesc& q, cudaStream_t s);
cudaError_t launch_finalize(const QueryDesc& q, cudaStream_t s);
cudaError_t launch_fold_sums(const QueryDesc& q, cudaStream_t s);
// rows of one fused-kernel launch: longer queries are split so that no global
// SUM limb word receives 2^31 or more additions between two folds
constexpr uint64_t kLaunchRows = 1ull << 31;
// segment mode walks run by run when the columns' entries (runs, twice the
// listed rows) average at least this many rows apart
constexpr uint64_t kRunWalkMinSegment = 64;
size_t query_kernel_smem(const QueryDesc& q);
cudaError_t query_kernel_set_smem(size_t bytes);

// batches (cq_batch.cu): the persistent kernel's static shared memory, its
// dynamic-size attribute, and the launch of init -> items -> finalize
cudaError_t batch_kernel_static_smem(int minb, size_t* bytes);
cudaError_t batch_kernel_set_smem(int minb, size_t bytes);
cudaError_t launch_batch(BatchCtl* ctl_dev, cudaStream_t s, unsigned grid, int minb, size_t dyn_smem,
                         unsigned aux_grid);

// planner / results (cq_api.cu)
int plan_batch_query(cq_table* table, const cq_plan* plan, uint32_t tile_rows, size_t smem_limit, Planned* P);
int plan_solo_query(cq_table* table, const cq_plan* plan, Planned* P);
int prepare_row_kernel(cq_ctx* ctx, Planned& P);
QueryBlock query_block_layout(const Planned& P, bool with_aux);
void bind_query_block(Planned& P, uint8_t* base, const QueryBlock& L, const uint32_t* aux_dev);
void attach_outputs(cq_result* r, const Planned& P);
cq_result* new_result(cq_ctx* ctx, cudaStream_t s, bool own_events);
int launch_solo(cq_table* table, Planned& P, cudaStream_t s, cq_result** out);
void free_result(cq_result* r);

// A plan whose filter is in conjunctive form (cq_filter.cu): `plan` is the
// input with a filter program replaced by `preds`, one entry per predicate
// occurrence with or_group / negate set; without a program, the input itself.
struct NormFilter {
  std::vector<cq_predicate> preds;
  cq_plan plan;
};
int normalize_filter(const cq_plan* in, NormFilter* out);

}  // namespace cq
