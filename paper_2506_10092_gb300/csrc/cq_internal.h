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

namespace cq {

// ---------------------------------------------------------------- limits
constexpr int kMaxCols = 16;      // referenced columns per query
constexpr int kMaxPreds = 16;
constexpr int kMaxKeys = 8;
constexpr int kMaxAggs = 16;
constexpr int kMaxBitmapCols = 8; // RLE / index columns per query
constexpr int kMaxPassBitmaps = 4; // row-mode predicates evaluated once per run
constexpr uint64_t kDenseMaxGroups = 1ull << 24;

enum Enc : uint8_t { ENC_RLE = 1, ENC_DICT = 2, ENC_INDEX = 3, ENC_PACKED = 4, ENC_PLAIN = 5 };

// Normalised predicate kinds.  Every comparison becomes an inclusive range
// or an inequality on the column's *raw* value: the logical value for RLE /
// index / plain columns, the unsigned field (code or offset) for dictionary
// and bit-packed columns (bit width < 64).
enum PredKind : uint8_t {
  PK_RANGE = 0,   // lo <= raw <= hi
  PK_NE = 1,      // raw != lo
  PK_BITMAP = 2,  // bit (raw - lo) of the aux bitmap; outside [lo, hi] fails
  PK_LIST = 3,    // raw in sorted aux list (binary search)
  PK_FALSE = 4,
  PK_TRUE = 5,
};

enum AggKind : uint8_t {
  AK_COUNT = 0,
  AK_SUM = 1,       // raw values (packed: offsets; finalize adds base * COUNT)
  AK_MIN = 2,
  AK_MAX = 3,
  AK_ISUM = 4,      // index column: sum of (value - default) over listed passing rows
  AK_IMIN = 5,      // index column: min over listed passing rows + listed count
  AK_IMAX = 6,
};

// Device view of one referenced column.
struct ColDesc {
  uint8_t enc;
  uint8_t v64;       // RLE/INDEX/PLAIN values are int64
  uint8_t e64;       // RLE ends / INDEX positions are int64
  uint8_t bw;        // PACKED/DICT bit width
  uint8_t bslot;     // RLE/INDEX: bitmap slot, 0xFF otherwise
  uint8_t raw_is_offset;  // PACKED with bw < 64: raw value is the unsigned offset
  uint16_t pad0;
  uint32_t stage_off;     // row-level columns: byte offset of the column inside a stage
  uint32_t stage_bytes;   // bytes staged per full tile
  int64_t base;      // PACKED base, INDEX default
  const void* vals;  // RLE run_values | PACKED/DICT words | INDEX values | PLAIN values
  const void* ends;  // RLE run_ends | INDEX positions
  uint64_t n;        // RLE n_runs | INDEX nnz | PACKED/DICT n_words | PLAIN n_rows
};

struct PredDesc {
  uint8_t col;       // index into QueryDesc::cols
  uint8_t kind;
  uint8_t n32;       // raw values and bounds fit int32: evaluate in 32 bits (lo32 / hi32)
  uint8_t pbm;       // row mode, RLE / index column: slot of the tile pass bitmap the helper
                     // warp fills once per run / listed row (0xFF: evaluated per row)
  uint32_t aux_off;  // 32-bit words into the aux area (bitmap or list of int64 as word pairs)
  uint32_t aux_len;  // bitmap words / list entries
  int32_t lo32, hi32;
  int64_t lo, hi;
};

struct KeyDesc {
  uint8_t col;
  uint8_t remap;     // 1: digit = rank of raw in a bitmap (IN-list) -- aux bitmap + prefix
  uint8_t n32;       // raw values read in 32 bits and |kmin| <= 2^30: digits in 32-bit arithmetic
  uint8_t pad0;
  uint32_t aux_off;  // bitmap words (remap)
  uint32_t aux_len;  // bitmap words (remap)
  uint32_t card;     // number of digit values
  uint64_t stride;   // gid = sum digit * stride
  int64_t kmin;      // digit = raw - kmin (remap: bitmap covers raw - kmin)
  uint32_t prefix_off; // remap: uint32 prefix popcounts per bitmap word in aux
  uint32_t list_off;   // remap: sorted raw values (int64 word pairs) for decoding ranks
};

struct AggDesc {
  uint8_t kind;
  uint8_t col;       // index into QueryDesc::cols (unused for COUNT)
  uint8_t sw;        // first 64-bit shared-memory accumulator word
  uint8_t wide;      // SUM accumulates 128-bit in shared memory (two words)
  uint8_t sw32;      // first 32-bit shared-memory accumulator word
  uint32_t gw;       // first global accumulator word
  uint8_t op;        // cq_agg_op (for finalize)
  uint8_t out_kind;  // 0 int64, 1 uint64, 2 double
  uint8_t red32;     // SUM: |raw| < 2^24 -> a warp batch (<= 128 values) is reduced in 32 bits
  uint8_t w32;       // MIN/MAX: raw values fit int32 -> 32-bit shared accumulator, warp-reduced
  uint8_t n32;       // values read in 32 bits (narrow column and red32 / w32)
  uint8_t s32;       // SUM: shared accumulator is one 32-bit word (sw32): 1 unsigned, 2 signed;
                     // the flush period keeps it from wrapping
  int64_t base;      // value added back at finalize (packed base or index default)
};

struct QueryDesc {
  uint64_t n_rows;
  uint64_t n_tiles;
  uint32_t tile_rows;
  uint8_t n_cols, n_preds, n_keys, n_aggs;
  uint8_t seg_mode;        // 1: every referenced column is RLE/index -> items are segments
  uint8_t n_bitmaps;       // RLE/INDEX columns with a per-tile bitmap
  uint8_t n_row_cols;      // columns staged per tile (row mode)
  uint8_t stages;
  uint8_t ncw;             // row mode shape: 16 = one CTA of 16 compute warps per SM, 8 = two such CTAs,
                           // 24 / 28 = one CTA of 24 / 28 compute warps (6144 / 7168-row tiles)
  uint32_t stage_bytes;    // bytes of one stage (all row-level columns)
  uint32_t table_slots;    // shared-memory group-table slots (power of two)
  uint8_t table_dense;     // 1: slot = gid (gid domain fits the table)
  uint8_t n_sw;            // 64-bit shared accumulator words per slot
  uint8_t n_sw32;          // 32-bit shared accumulator words per slot (word 0 = COUNT)
  uint8_t n_gw;            // global accumulator words per group (word 0 = COUNT)
  uint8_t has_index_agg;
  uint8_t n_pbm;           // tile pass bitmaps: predicates 0 .. n_pbm-1 (row mode, RLE / index columns)
  uint32_t flush_rows;     // flush the shared table at least this often (rows)
  uint64_t n_groups;       // dense global domain
  uint8_t row_cols[kMaxCols];   // ColDesc indices of staged columns
  ColDesc cols[kMaxCols];
  PredDesc preds[kMaxPreds];
  KeyDesc keys[kMaxKeys];
  AggDesc aggs[kMaxAggs];
  const uint32_t* aux;     // device: bitmaps, prefix counts, sorted lists
  uint32_t aux_words;
  uint32_t smem_bytes;     // dynamic shared memory of the fused kernel
  // global state
  unsigned long long* gacc;  // [n_gw][n_groups]
  int* err;                  // device status word (cq_status, 0 = ok)
  unsigned long long* err_info;  // what / where / value of the first device error
  // outputs
  uint32_t n_out;
  uint8_t out_is_key[kMaxKeys + kMaxAggs];
  uint8_t out_index[kMaxKeys + kMaxAggs];
  void* out[kMaxKeys + kMaxAggs];  // device columns [n_groups capacity]
  unsigned long long* out_count;   // number of result rows
  unsigned int* block_counts;      // finalize scratch
};

// ---------------------------------------------------------------- batches
// One unit of a batch's work list: tiles [t_begin, t_begin + n_tiles) of query
// `query`.  A persistent kernel's CTAs take items in list order.
struct BatchItem {
  uint32_t query;
  uint32_t n_tiles;
  uint64_t t_begin;
};

// Header of a batch's control block (device memory, uploaded per launch):
// counts, the work counter and the arrays that follow the header.
struct BatchCtl {
  uint32_t n_queries;
  uint32_t n_items;
  uint32_t n_init_blocks;              // init blocks of all queries (kInitGroups groups each)
  uint32_t n_fin_blocks;               // finalize blocks of all queries (1024 groups each)
  unsigned long long next_item;        // work counter, 0 at upload
  const QueryDesc* descs;              // [n_queries]
  const BatchItem* items;              // [n_items], larger items first
  const uint32_t* init_first;          // [n_queries + 1] first init block of each query
  const uint32_t* fin_first;           // [n_queries + 1] first finalize block of each query
};

constexpr uint32_t kInitGroups = 1024;  // groups initialised per batch init block

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
};

// Byte offsets of one query's device buffers inside one allocation.
struct QueryBlock {
  uint64_t gacc, out, aux, err, cnt, blk, total;
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

// kernels / launchers (cq_query.cu)
cudaError_t launch_query(const QueryDesc& q, cudaStream_t s, int num_sms, int ctas_per_sm, uint32_t grid_ctas);
cudaError_t launch_init_global(const QueryDesc& q, cudaStream_t s);
cudaError_t launch_finalize(const QueryDesc& q, cudaStream_t s);
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
QueryBlock query_block_layout(const Planned& P, bool with_aux);
void bind_query_block(Planned& P, uint8_t* base, const QueryBlock& L, const uint32_t* aux_dev);
void attach_outputs(cq_result* r, const Planned& P);
cq_result* new_result(cq_ctx* ctx, cudaStream_t s, bool own_events);
int launch_solo(cq_table* table, Planned& P, cudaStream_t s, cq_result** out);
void free_result(cq_result* r);

}  // namespace cq
