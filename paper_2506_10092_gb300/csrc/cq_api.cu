// cq_api.cu -- the C ABI of include/cq.h: handles, validation, the query
// planner and the launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "cq_internal.h"

namespace cq {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int set_error(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return status;
}

void clear_error() { g_err.clear(); }

// kernels (cq_columns.cu / cq_query.cu)
cudaError_t run_column_check(const cq_column* c, void* d_out, cudaStream_t s);
cudaError_t align_segments(cq_column* const* cols, uint32_t k, cudaStream_t s, void* scratch_counts,
                           unsigned long long n_tiles, unsigned long long n_rows, long long* seg_ends,
                           long long* ridx, unsigned long long capacity, unsigned long long* host_counts,
                           unsigned long long* n_segments);
cudaError_t expand_column(const cq_column* c, long long* out, cudaStream_t s, int num_sms);

// ------------------------------------------------------------------ helpers
typedef __int128 i128;

long long fault_inject_at(const char* kind) {
  const char* v = getenv("CQ_FAULT_INJECT");
  const size_t n = strlen(kind);
  return (v && strncmp(v, kind, n) == 0 && v[n] == ':') ? atoll(v + n + 1) : 0ll;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s) {
  static const long long fail_at = fault_inject_at("alloc");
  static std::atomic<long long> calls{0};
  if (fail_at > 0 && ++calls == fail_at) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

static int cmp_bytes(const char* a, size_t la, const char* b, size_t lb) {
  const size_t m = la < lb ? la : lb;
  const int c = m ? memcmp(a, b, m) : 0;
  if (c) return c < 0 ? -1 : 1;
  return la == lb ? 0 : (la < lb ? -1 : 1);
}

static bool dtype_ok(int t) { return t == CQ_I32 || t == CQ_I64; }
static size_t dsize(int t) { return t == CQ_I64 ? 8 : 4; }

static uint64_t pad16(uint64_t bytes) { return (bytes + 15) / 16 * 16; }

// Allocate library-owned device memory (padded to 16 bytes plus 16 of slack)
// from the context's stream-ordered pool and fill it from host or device
// memory; only the padding is cleared.  The column's creation synchronises
// the context's stream before the buffer is used anywhere else.
static int own_copy(cq_ctx* ctx, const void* src, uint64_t bytes, bool from_device, void** dst) {
  const uint64_t alloc = pad16(bytes) + 16;
  void* p = nullptr;
  if (pool_alloc((void**)&p, alloc, ctx->pool, ctx->stream) != cudaSuccess)
    return set_error(CQ_ERR_OOM, "device allocation of %llu bytes failed", (unsigned long long)alloc);
  cudaMemsetAsync(reinterpret_cast<uint8_t*>(p) + bytes, 0, alloc - bytes, ctx->stream);
  if (bytes) {
    cudaError_t e = cudaMemcpyAsync(p, src, bytes, from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(p, ctx->stream);
      return set_error(CQ_ERR_CUDA, "copy of column buffer failed: %s", cudaGetErrorString(e));
    }
  }
  *dst = p;
  return CQ_OK;
}

static int check_borrow(const void* p, const char* what) {
  if (p && (reinterpret_cast<uintptr_t>(p) & 15))
    return set_error(CQ_ERR_INVALID_ARG, "borrowed %s buffer is not 16-byte aligned", what);
  return CQ_OK;
}

// Validate on the device and record the column's raw / logical ranges.
static int finish_column(cq_column* c) {
  cq_ctx* ctx = c->ctx;
  void* d = nullptr;
  CQ_CUDA(pool_alloc((void**)&d, 64, ctx->pool, ctx->stream));
  struct {
    int err, pad;
    long long mn, mx;
  } h{};
  cudaError_t e = run_column_check(c, d, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(d, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "column check failed: %s", cudaGetErrorString(e));
  if (h.err) {
    const char* why = h.err == CQ_ERR_UNSORTED ? "run ends / positions are not strictly increasing"
                      : h.err == CQ_ERR_SIZE_MISMATCH ? "last run end differs from n_rows"
                      : c->enc == ENC_DICT ? "a code is not below the dictionary size"
                                           : "a position is out of range";
    return set_error(h.err, "column rejected: %s", why);
  }
  ColumnStats& st = c->stats;
  const bool empty = h.mx < h.mn;
  st.min_raw = empty ? 0 : h.mn;
  st.max_raw = empty ? -1 : h.mx;
  i128 lo = st.min_raw, hi = st.max_raw;
  if (c->enc == ENC_PACKED) {
    lo += c->base;
    hi += c->base;
    if (c->bit_width == 64) {  // 64-bit fields: raw range is already the logical value's
      lo = (i128)st.min_raw + (i128)c->base;
      hi = (i128)st.max_raw + (i128)c->base;
    }
  }
  if (c->enc == ENC_INDEX && c->n < c->n_rows) {
    if (empty) { lo = hi = c->base; }
    else { lo = std::min(lo, (i128)c->base); hi = std::max(hi, (i128)c->base); }
  }
  const bool fits = lo >= (i128)LLONG_MIN && hi <= (i128)LLONG_MAX;
  st.min_val = fits ? (int64_t)lo : LLONG_MIN;
  st.max_val = fits ? (int64_t)hi : LLONG_MAX;
  const i128 a = std::max(lo < 0 ? -lo : lo, hi < 0 ? -hi : hi);
  st.max_abs_val = a > (i128)ULLONG_MAX ? ULLONG_MAX : (uint64_t)a;
  if (c->enc == ENC_INDEX && c->n == c->n_rows && empty) st.max_abs_val = 0;
  return CQ_OK;
}

}  // namespace cq

using namespace cq;

// ====================================================================== context
extern "C" const char* cq_last_error(void) { return g_err.c_str(); }

extern "C" int cq_ctx_create(int device, void* cuda_stream, cq_ctx** out) {
  clear_error();
  if (!out) return set_error(CQ_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0)
    return set_error(CQ_ERR_CUDA, "no CUDA device is available (this library has no CPU path)");
  if (device < 0 || device >= n) return set_error(CQ_ERR_INVALID_ARG, "device %d out of range", device);
  CQ_CUDA(cudaSetDevice(device));
  std::unique_ptr<cq_ctx> c(new cq_ctx);
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  CQ_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  int smem = 0;
  CQ_CUDA(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  c->smem_optin = (size_t)smem;
  int per_sm = 0, reserved = 0;
  CQ_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  CQ_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
  c->smem_two = (size_t)(per_sm / 2 - reserved);
  c->smem_three = (size_t)(per_sm / 3 - reserved) / 128 * 128;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  CQ_CUDA(cudaMemPoolCreate(&c->pool, &props));
  uint64_t thr = UINT64_MAX;
  CQ_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr));
  CQ_CUDA(query_kernel_set_smem(c->smem_optin));
  *out = c.release();
  return CQ_OK;
}

namespace cq {
void ctx_release(cq_ctx* ctx) {
  if (--ctx->refs > 0) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (!ctx->graphs.empty()) cudaDeviceSynchronize();   // batch graphs may still be running
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

void clear_stale_error(const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    static const bool dbg = getenv("CQ_DEBUG") != nullptr;
    if (dbg) fprintf(stderr, "cq: stale CUDA error before %s: %s\n", where, cudaGetErrorString(e));
  }
}
}  // namespace cq

cq_column::~cq_column() {
  if (ctx) ctx_release(ctx);
}

// The context lives on while columns created in it do (tables and results
// hold their columns), whatever order the handles are destroyed in.
extern "C" int cq_ctx_destroy(cq_ctx* ctx) {
  clear_error();
  if (!ctx) return CQ_OK;
  ctx_release(ctx);
  return CQ_OK;
}

extern "C" int cq_ctx_num_sms(cq_ctx* ctx, uint32_t* out) {
  if (!ctx || !out) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *out = (uint32_t)ctx->num_sms;
  return CQ_OK;
}

// ====================================================================== columns
static int new_column(cq_ctx* ctx, uint8_t enc, uint64_t n_rows, cq_column** out, std::unique_ptr<cq_column>* c) {
  if (!ctx || !out) return set_error(CQ_ERR_INVALID_ARG, "NULL context or out");
  *out = nullptr;
  c->reset(new cq_column);
  (*c)->ctx = ctx;
  ctx->refs++;
  (*c)->enc = enc;
  (*c)->n_rows = n_rows;
  CQ_CUDA(cudaSetDevice(ctx->device));
  return CQ_OK;
}

// Owned buffers go back to the context's pool (every query that used them
// has finished: results hold their columns until their stream is drained).
static void release_buffers(cq_column* c) {
  if (c->owned) {
    if (c->vals) cudaFreeAsync(c->vals, c->ctx->stream);
    if (c->ends) cudaFreeAsync(c->ends, c->ctx->stream);
  }
  c->vals = c->ends = nullptr;
}

static int finish_or_release(std::unique_ptr<cq_column>& c, cq_column** out) {
  int rc = finish_column(c.get());
  if (rc != CQ_OK) {
    release_buffers(c.get());
    return rc;
  }
  *out = c.release();
  return CQ_OK;
}

extern "C" int cq_column_create_rle(cq_ctx* ctx, cq_dtype val_t, const void* run_values, cq_dtype end_t,
                                    const void* run_ends, uint64_t n_runs, uint64_t n_rows, uint32_t mem_flags,
                                    cq_column** out) {
  clear_error();
  std::unique_ptr<cq_column> c;
  int rc = new_column(ctx, ENC_RLE, n_rows, out, &c);
  if (rc) return rc;
  if (!dtype_ok(val_t) || !dtype_ok(end_t)) return set_error(CQ_ERR_INVALID_ARG, "bad dtype");
  if (n_rows > 0 && n_runs == 0) return set_error(CQ_ERR_SIZE_MISMATCH, "no runs for %llu rows", (unsigned long long)n_rows);
  if (n_rows == 0 && n_runs != 0) return set_error(CQ_ERR_SIZE_MISMATCH, "runs given for an empty column");
  if (end_t == CQ_I32 && n_rows > (uint64_t)INT_MAX) return set_error(CQ_ERR_INVALID_ARG, "int32 run ends cannot address n_rows");
  if (n_runs && (!run_values || !run_ends)) return set_error(CQ_ERR_INVALID_ARG, "NULL buffer");
  c->val_t = val_t;
  c->end_t = end_t;
  c->n = n_runs;
  if (mem_flags == CQ_MEM_DEVICE_BORROW) {
    if ((rc = check_borrow(run_values, "run_values")) || (rc = check_borrow(run_ends, "run_ends"))) return rc;
    c->vals = const_cast<void*>(run_values);
    c->ends = const_cast<void*>(run_ends);
  } else {
    c->owned = true;
    if ((rc = own_copy(ctx, run_values, n_runs * dsize(val_t), false, &c->vals))) return rc;
    if ((rc = own_copy(ctx, run_ends, n_runs * dsize(end_t), false, &c->ends))) { release_buffers(c.get()); return rc; }
  }
  c->device_bytes = n_runs * (dsize(val_t) + dsize(end_t));
  return finish_or_release(c, out);
}

// RLE + Index composite (Section 3.2).  The runs and the listed rows are
// merged in row order into one RLE column whose unit runs are the listed
// rows: here a run costs a value and an end, as a listed row costs a value
// and a position, so the merged column is as large as the composite.
extern "C" int cq_column_create_rle_index(cq_ctx* ctx, cq_dtype val_t, cq_dtype pos_t, const void* run_values,
                                          const void* run_starts, const void* run_ends, uint64_t n_runs,
                                          const void* values, const void* positions, uint64_t nnz, uint64_t n_rows,
                                          cq_column** out) {
  clear_error();
  if (!ctx || !out) return set_error(CQ_ERR_INVALID_ARG, "NULL context or output");
  if (!dtype_ok(val_t) || !dtype_ok(pos_t)) return set_error(CQ_ERR_INVALID_ARG, "bad dtype");
  if ((n_runs && (!run_values || !run_starts || !run_ends)) || (nnz && (!values || !positions)))
    return set_error(CQ_ERR_INVALID_ARG, "NULL buffer");
  auto rd = [](const void* p, cq_dtype t, uint64_t i) -> int64_t {
    return t == CQ_I32 ? (int64_t) static_cast<const int32_t*>(p)[i] : static_cast<const int64_t*>(p)[i];
  };
  std::vector<int64_t> mv, me;
  mv.reserve(n_runs + nnz);
  me.reserve(n_runs + nnz);
  // rows in order: the next row must start a run or be listed
  uint64_t cursor = 0, i = 0, k = 0;
  while (i < n_runs || k < nnz) {
    if (i < n_runs && rd(run_starts, pos_t, i) == (int64_t)cursor) {
      const int64_t e = rd(run_ends, pos_t, i);
      if (e <= (int64_t)cursor)
        return set_error(CQ_ERR_UNSORTED, "run %llu is empty or ends before it starts", (unsigned long long)i);
      mv.push_back(rd(run_values, val_t, i));
      me.push_back(e);
      cursor = (uint64_t)e;
      ++i;
    } else if (k < nnz && rd(positions, pos_t, k) == (int64_t)cursor) {
      mv.push_back(rd(values, val_t, k));
      me.push_back((int64_t)cursor + 1);
      ++cursor;
      ++k;
    } else {
      return set_error(CQ_ERR_SIZE_MISMATCH,
                       "row %llu is neither the start of the next run nor the next listed row (a gap, an overlap "
                       "or unsorted input)", (unsigned long long)cursor);
    }
    if (cursor > n_rows)
      return set_error(CQ_ERR_SIZE_MISMATCH, "runs and listed rows reach past n_rows %llu", (unsigned long long)n_rows);
  }
  if (cursor != n_rows)
    return set_error(CQ_ERR_SIZE_MISMATCH, "runs and listed rows cover %llu of %llu rows", (unsigned long long)cursor,
                     (unsigned long long)n_rows);
  // the RLE column keeps the value type; ends in 32 bits when they fit
  std::vector<int32_t> v32, e32;
  const void* vp = mv.data();
  const void* ep = me.data();
  if (val_t == CQ_I32) {
    v32.assign(mv.begin(), mv.end());
    vp = v32.data();
  }
  const cq_dtype end_t = n_rows <= (uint64_t)INT_MAX ? CQ_I32 : CQ_I64;
  if (end_t == CQ_I32) {
    e32.assign(me.begin(), me.end());
    ep = e32.data();
  }
  return cq_column_create_rle(ctx, val_t, vp, end_t, ep, mv.size(), n_rows, CQ_MEM_HOST_COPY, out);
}

extern "C" int cq_column_create_dict(cq_ctx* ctx, const char* dict_bytes, const uint64_t* dict_offsets,
                                     uint32_t n_entries, const uint32_t* packed_codes, uint64_t n_words,
                                     uint32_t bit_width, uint64_t n_rows, uint32_t mem_flags, cq_column** out) {
  clear_error();
  std::unique_ptr<cq_column> c;
  int rc = new_column(ctx, ENC_DICT, n_rows, out, &c);
  if (rc) return rc;
  if (bit_width < 1 || bit_width > 32) return set_error(CQ_ERR_INVALID_ARG, "dictionary code width %u not in 1..32", bit_width);
  if (n_entries == 0 && n_rows > 0) return set_error(CQ_ERR_INVALID_ARG, "empty dictionary");
  if (n_entries && (!dict_bytes || !dict_offsets)) return set_error(CQ_ERR_INVALID_ARG, "NULL dictionary");
  const uint64_t need = (n_rows * bit_width + 31) / 32;
  const uint64_t need_pad = (need + 3) / 4 * 4;
  if (n_words < need) return set_error(CQ_ERR_INVALID_ARG, "%llu code words given, %llu needed", (unsigned long long)n_words, (unsigned long long)need);
  if (mem_flags == CQ_MEM_DEVICE_BORROW && n_words < need_pad)
    return set_error(CQ_ERR_INVALID_ARG, "borrowed code words must be padded to %llu words", (unsigned long long)need_pad);
  c->n_entries = n_entries;
  c->dict_offsets.assign(dict_offsets, dict_offsets + (n_entries ? n_entries + 1 : 0));
  if (n_entries) {
    if (dict_offsets[0] != 0) return set_error(CQ_ERR_INVALID_ARG, "dictionary offsets must start at 0");
    for (uint32_t i = 0; i < n_entries; ++i)
      if (dict_offsets[i + 1] < dict_offsets[i]) return set_error(CQ_ERR_INVALID_ARG, "dictionary offsets decrease");
    c->dict_bytes.assign(dict_bytes, dict_bytes + dict_offsets[n_entries]);
    for (uint32_t i = 0; i + 1 < n_entries; ++i) {
      const char* a = c->dict_bytes.data() + dict_offsets[i];
      const char* b = c->dict_bytes.data() + dict_offsets[i + 1];
      if (cmp_bytes(a, dict_offsets[i + 1] - dict_offsets[i], b, dict_offsets[i + 2] - dict_offsets[i + 1]) >= 0)
        return set_error(CQ_ERR_INVALID_ARG, "dictionary is not sorted and unique at entry %u", i);
    }
  }
  c->bit_width = bit_width;
  c->n = n_words;
  if (mem_flags == CQ_MEM_DEVICE_BORROW) {
    if ((rc = check_borrow(packed_codes, "packed_codes"))) return rc;
    c->vals = const_cast<uint32_t*>(packed_codes);
  } else {
    c->owned = true;
    if ((rc = own_copy(ctx, packed_codes, need * 4, false, &c->vals))) return rc;
    c->n = (pad16(need * 4) + 16) / 4;
  }
  c->device_bytes = (n_rows * bit_width + 7) / 8;
  return finish_or_release(c, out);
}

extern "C" int cq_column_create_index(cq_ctx* ctx, cq_dtype val_t, const void* values, cq_dtype pos_t,
                                      const void* positions, uint64_t nnz, int64_t default_value, uint64_t n_rows,
                                      uint32_t mem_flags, cq_column** out) {
  clear_error();
  std::unique_ptr<cq_column> c;
  int rc = new_column(ctx, ENC_INDEX, n_rows, out, &c);
  if (rc) return rc;
  if (!dtype_ok(val_t) || !dtype_ok(pos_t)) return set_error(CQ_ERR_INVALID_ARG, "bad dtype");
  if (nnz > n_rows) return set_error(CQ_ERR_INVALID_ARG, "more listed positions than rows");
  if (nnz && (!values || !positions)) return set_error(CQ_ERR_INVALID_ARG, "NULL buffer");
  c->val_t = val_t;
  c->end_t = pos_t;
  c->n = nnz;
  c->base = default_value;
  if (mem_flags == CQ_MEM_DEVICE_BORROW) {
    if ((rc = check_borrow(values, "values")) || (rc = check_borrow(positions, "positions"))) return rc;
    c->vals = const_cast<void*>(values);
    c->ends = const_cast<void*>(positions);
  } else {
    c->owned = true;
    if ((rc = own_copy(ctx, values, nnz * dsize(val_t), false, &c->vals))) return rc;
    if ((rc = own_copy(ctx, positions, nnz * dsize(pos_t), false, &c->ends))) { release_buffers(c.get()); return rc; }
  }
  c->device_bytes = nnz * (dsize(val_t) + dsize(pos_t));
  return finish_or_release(c, out);
}

extern "C" int cq_column_create_bitpacked(cq_ctx* ctx, cq_dtype logical_t, const uint32_t* words, uint64_t n_words,
                                          uint32_t bit_width, int64_t base, uint64_t n_rows, uint32_t mem_flags,
                                          cq_column** out) {
  clear_error();
  std::unique_ptr<cq_column> c;
  int rc = new_column(ctx, ENC_PACKED, n_rows, out, &c);
  if (rc) return rc;
  if (!dtype_ok(logical_t)) return set_error(CQ_ERR_INVALID_ARG, "bad dtype");
  if (bit_width < 1 || bit_width > 64) return set_error(CQ_ERR_INVALID_ARG, "bit width %u not in 1..64", bit_width);
  const uint64_t need = (n_rows * bit_width + 31) / 32;
  const uint64_t need_pad = (need + 3) / 4 * 4;
  if (n_words < need) return set_error(CQ_ERR_INVALID_ARG, "%llu words given, %llu needed", (unsigned long long)n_words, (unsigned long long)need);
  if (mem_flags == CQ_MEM_DEVICE_BORROW && n_words < need_pad)
    return set_error(CQ_ERR_INVALID_ARG, "borrowed words must be padded to %llu words", (unsigned long long)need_pad);
  c->logical_t = logical_t;
  c->bit_width = bit_width;
  c->base = base;
  c->n = n_words;
  if (mem_flags == CQ_MEM_DEVICE_BORROW) {
    if ((rc = check_borrow(words, "words"))) return rc;
    c->vals = const_cast<uint32_t*>(words);
  } else {
    c->owned = true;
    if ((rc = own_copy(ctx, words, need * 4, false, &c->vals))) return rc;
    c->n = (pad16(need * 4) + 16) / 4;
  }
  c->device_bytes = (n_rows * bit_width + 7) / 8;
  return finish_or_release(c, out);
}

extern "C" int cq_column_create_plain(cq_ctx* ctx, cq_dtype t, const void* values, uint64_t n_rows,
                                      uint32_t mem_flags, cq_column** out) {
  clear_error();
  std::unique_ptr<cq_column> c;
  int rc = new_column(ctx, ENC_PLAIN, n_rows, out, &c);
  if (rc) return rc;
  if (!dtype_ok(t)) return set_error(CQ_ERR_INVALID_ARG, "bad dtype");
  if (n_rows && !values) return set_error(CQ_ERR_INVALID_ARG, "NULL buffer");
  c->val_t = t;
  c->n = n_rows;
  if (mem_flags == CQ_MEM_DEVICE_BORROW) {
    if ((rc = check_borrow(values, "values"))) return rc;
    c->vals = const_cast<void*>(values);
  } else {
    c->owned = true;
    if ((rc = own_copy(ctx, values, n_rows * dsize(t), false, &c->vals))) return rc;
  }
  c->device_bytes = n_rows * dsize(t);
  return finish_or_release(c, out);
}

extern "C" int cq_column_destroy(cq_column* col) {
  clear_error();
  if (!col) return CQ_OK;
  if (--col->refs == 0) {
    cudaSetDevice(col->ctx->device);
    cudaStreamSynchronize(col->ctx->stream);
    release_buffers(col);
    delete col;
  }
  return CQ_OK;
}

extern "C" int cq_column_encoding(const cq_column* col, uint32_t* enc) {
  if (!col || !enc) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *enc = col->enc;
  return CQ_OK;
}

extern "C" int cq_column_device_bytes(const cq_column* col, uint64_t* bytes) {
  if (!col || !bytes) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *bytes = col->device_bytes;
  return CQ_OK;
}

// ====================================================================== tables
extern "C" int cq_table_bind(cq_ctx* ctx, cq_column* const* cols, uint32_t n_cols, cq_table** out) {
  clear_error();
  if (!ctx || !out || (n_cols && !cols)) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_cols == 0) return set_error(CQ_ERR_INVALID_ARG, "a table needs at least one column");
  for (uint32_t i = 0; i < n_cols; ++i) {
    if (!cols[i]) return set_error(CQ_ERR_INVALID_ARG, "column %u is NULL", i);
    if (cols[i]->ctx != ctx) return set_error(CQ_ERR_INVALID_ARG, "column %u belongs to another context", i);
    if (cols[i]->n_rows != cols[0]->n_rows)
      return set_error(CQ_ERR_SIZE_MISMATCH, "column %u has %llu rows, column 0 has %llu", i,
                       (unsigned long long)cols[i]->n_rows, (unsigned long long)cols[0]->n_rows);
  }
  cq_table* t = new cq_table;
  t->ctx = ctx;
  t->n_rows = cols[0]->n_rows;
  for (uint32_t i = 0; i < n_cols; ++i) {
    cols[i]->refs++;
    t->cols.push_back(cols[i]);
  }
  *out = t;
  return CQ_OK;
}

extern "C" int cq_table_destroy(cq_table* table) {
  clear_error();
  if (!table) return CQ_OK;
  for (cq_column* c : table->cols) cq_column_destroy(c);
  delete table;
  return CQ_OK;
}

extern "C" int cq_table_num_rows(const cq_table* table, uint64_t* n_rows) {
  if (!table || !n_rows) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *n_rows = table->n_rows;
  return CQ_OK;
}

// ====================================================================== planner
namespace cq {

// A column as the planner sees it (a table column, or the flat int64 array
// the decompress-then-scan path expanded it to).
struct PlanCol {
  uint8_t enc;
  bool v64, e64;
  uint32_t bw;
  int64_t base;
  const void* vals;
  const void* ends;
  uint64_t n;
  ColumnStats stats;
  const cq_column* src;   // dictionary and key-string lookups
};

static PlanCol view_of(const cq_column* c) {
  PlanCol p;
  p.enc = c->enc;
  p.v64 = c->val_t == CQ_I64;
  p.e64 = c->end_t == CQ_I64;
  p.bw = c->bit_width;
  p.base = c->base;
  p.vals = c->vals;
  p.ends = c->ends;
  p.n = c->n;
  p.stats = c->stats;
  p.src = c;
  return p;
}

static bool is_dict(const PlanCol& c) { return c.src && c.src->enc == ENC_DICT; }

// lower / upper bound of a literal in the sorted dictionary
static uint32_t dict_bound(const cq_column* d, const char* s, size_t ls, bool upper) {
  uint32_t lo = 0, hi = d->n_entries;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) / 2;
    const char* m = d->dict_bytes.data() + d->dict_offsets[mid];
    const size_t lm = d->dict_offsets[mid + 1] - d->dict_offsets[mid];
    const int c = cmp_bytes(m, lm, s, ls);
    if (c < 0 || (upper && c == 0)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

static size_t lit_len(const cq_predicate& p, uint32_t i) {
  return p.str_lens ? p.str_lens[i] : strlen(p.strs[i]);
}

// Raw-space transform of a logical integer interval for one column.
struct RawMap {
  bool offset;       // raw = logical - base (bit-packed, no wrap-around)
  int64_t base;
  i128 rmin, rmax;   // raw domain
};

static RawMap raw_map(const PlanCol& c, bool raw_is_offset) {
  RawMap m;
  m.offset = raw_is_offset;
  m.base = raw_is_offset ? c.base : 0;
  if (raw_is_offset) {
    m.rmin = 0;
    m.rmax = (((i128)1) << c.bw) - 1;
  } else {
    m.rmin = LLONG_MIN;
    m.rmax = LLONG_MAX;
  }
  return m;
}

static void set_range(PredDesc& d, i128 lo, i128 hi, const RawMap& m) {
  lo -= m.base;
  hi -= m.base;
  if (lo < m.rmin) lo = m.rmin;
  if (hi > m.rmax) hi = m.rmax;
  if (lo > hi) {
    d.kind = PK_FALSE;
    return;
  }
  d.kind = PK_RANGE;
  d.lo = (int64_t)lo;
  d.hi = (int64_t)hi;
}

// Bitmap (small span) or sorted list of raw values in aux.
static void set_members(PredDesc& d, std::vector<int64_t> vals, std::vector<uint32_t>& aux) {
  std::sort(vals.begin(), vals.end());
  vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
  if (vals.empty()) {
    d.kind = PK_FALSE;
    return;
  }
  const i128 span = (i128)vals.back() - (i128)vals.front();
  if (span < (1 << 20)) {
    const uint32_t words = (uint32_t)(span / 32 + 1);
    d.kind = PK_BITMAP;
    d.lo = vals.front();
    d.hi = vals.back();
    d.aux_off = (uint32_t)aux.size();
    d.aux_len = words;
    aux.resize(aux.size() + words, 0u);
    for (int64_t v : vals) {
      const uint64_t o = (uint64_t)((i128)v - (i128)d.lo);
      aux[d.aux_off + o / 32] |= 1u << (o % 32);
    }
  } else {
    d.kind = PK_LIST;
    if (aux.size() & 1) aux.push_back(0);  // 8-byte alignment of the list
    d.aux_off = (uint32_t)aux.size();
    d.aux_len = (uint32_t)vals.size();
    for (int64_t v : vals) {
      aux.push_back((uint32_t)(uint64_t)v);
      aux.push_back((uint32_t)((uint64_t)v >> 32));
    }
  }
}

// Capacity of a query's global hash table: 2^lg slots, and the CTAs of its
// finalize sort (about 4096 slots each, at most 1024).
static void set_hash_capacity(QueryDesc& q, uint32_t lg) {
  q.n_groups = 1ull << lg;
  const uint64_t b = q.n_groups / 4096;
  q.sort_blocks = (uint32_t)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

static int plan_query_tile(const std::vector<PlanCol>& tcols, uint64_t n_rows, const cq_plan* plan,
                           const cq_exec_options* opts, const cq_ctx* ctx, uint32_t tile, int ncw,
                           size_t smem_limit, Planned* P, bool* no_fit, bool batch) {
  *no_fit = false;
  if (!plan) return set_error(CQ_ERR_INVALID_ARG, "plan is NULL");
  if (plan->n_preds > (uint32_t)kMaxPreds || plan->n_group_by > (uint32_t)kMaxKeys || plan->n_aggs > (uint32_t)kMaxAggs)
    return set_error(CQ_ERR_INVALID_ARG, "plan exceeds 16 predicates / 8 group-by columns / 16 aggregates");
  if ((plan->n_preds && !plan->preds) || (plan->n_group_by && !plan->group_by) || (plan->n_aggs && !plan->aggs))
    return set_error(CQ_ERR_INVALID_ARG, "plan array is NULL");
  QueryDesc& q = P->q;
  memset(&q, 0, sizeof(q));
  q.n_rows = n_rows;
  std::vector<int> slot(tcols.size(), -1);
  std::vector<int> order;
  auto use = [&](uint32_t col) -> int {
    if (col >= tcols.size()) return -1;
    if (slot[col] < 0) {
      if (order.size() >= (size_t)kMaxCols) return -2;
      slot[col] = (int)order.size();
      order.push_back((int)col);
    }
    return slot[col];
  };
  for (uint32_t i = 0; i < plan->n_preds; ++i)
    if (use(plan->preds[i].col) < 0) return set_error(CQ_ERR_INVALID_ARG, "predicate %u: bad column %u", i, plan->preds[i].col);
  for (uint32_t i = 0; i < plan->n_group_by; ++i)
    if (use(plan->group_by[i]) < 0) return set_error(CQ_ERR_INVALID_ARG, "group-by %u: bad column %u", i, plan->group_by[i]);
  for (uint32_t i = 0; i < plan->n_aggs; ++i) {
    const cq_aggregate& a = plan->aggs[i];
    if (a.op < CQ_SUM || a.op > CQ_STD_SAMP) return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: bad op %d", i, a.op);
    if (a.op == CQ_COUNT) continue;
    if (use(a.col) < 0) return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: bad column %u", i, a.col);
    if (a.op != CQ_MIN && a.op != CQ_MAX && is_dict(tcols[a.col]))
      return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: SUM/AVG/VAR/STD of a dictionary column", i);
    if (a.expr < CQ_EXPR_NONE || a.expr > CQ_EXPR_MUL)
      return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: bad expression %d", i, a.expr);
    if (a.expr != CQ_EXPR_NONE) {
      if (a.op != CQ_SUM && a.op != CQ_MIN && a.op != CQ_MAX && a.op != CQ_AVG)
        return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: expressions take SUM, MIN, MAX and AVG", i);
      if (use(a.col2) < 0) return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: bad column %u", i, a.col2);
      if (is_dict(tcols[a.col]) || is_dict(tcols[a.col2]))
        return set_error(CQ_ERR_INVALID_ARG, "aggregate %u: expression over a dictionary column", i);
    }
  }
  // ---- tile / pipeline shape
  q.tile_rows = tile;
  q.n_tiles = (n_rows + tile - 1) / tile;
  q.n_cols = (uint8_t)order.size();
  // ---- columns
  int nb = 0, nrow = 0;
  uint32_t stage_off = 0;
  for (size_t i = 0; i < order.size(); ++i) {
    const PlanCol& pc = tcols[order[i]];
    ColDesc& d = q.cols[i];
    d.enc = pc.enc;
    d.v64 = pc.v64;
    d.e64 = pc.e64;
    d.bw = (uint8_t)pc.bw;
    d.base = pc.base;
    d.vals = pc.vals;
    d.ends = pc.ends;
    d.n = pc.n;
    d.bslot = 0xFF;
    d.raw_is_offset = 0;
    if (pc.enc == ENC_DICT) d.raw_is_offset = 1;
    if (pc.enc == ENC_PACKED && pc.bw < 64 && (i128)pc.base + ((((i128)1) << pc.bw) - 1) <= (i128)LLONG_MAX)
      d.raw_is_offset = 1;
    if (pc.enc == ENC_RLE || pc.enc == ENC_INDEX) {
      if (nb >= kMaxBitmapCols) return set_error(CQ_ERR_UNSUPPORTED, "more than %d RLE / index columns in one query", kMaxBitmapCols);
      d.bslot = (uint8_t)nb++;
    } else {
      const uint32_t bits = pc.enc == ENC_PLAIN ? (pc.v64 ? 64u : 32u) : pc.bw;
      d.stage_off = stage_off;
      d.stage_bytes = (uint32_t)(pad16((uint64_t)tile * bits / 8) + 16);
      stage_off += d.stage_bytes;
      q.row_cols[nrow++] = (uint8_t)i;
    }
  }
  q.n_bitmaps = (uint8_t)nb;
  q.n_row_cols = (uint8_t)nrow;
  q.seg_mode = nrow == 0;
  // segment mode walks tile by tile (bitmaps of the boundaries) or, when the
  // segments are long, run by run (a merge of the columns' boundaries whose
  // work follows the runs): kernel option 2 / 3 pins one
  q.run_walk = 0;
  q.run_slot = 0;
  if (q.seg_mode && nb > 0 && !batch) {
    uint64_t entries = 0, most = 0;
    for (int c = 0; c < q.n_cols; ++c) {
      const ColDesc& d = q.cols[c];
      if (d.bslot == 0xFF) continue;
      entries += d.enc == ENC_INDEX ? 2 * d.n : d.n;
      if (d.n >= most) {
        most = d.n;
        q.run_slot = d.bslot;
      }
    }
    const uint32_t k = opts ? opts->kernel : 0;
    q.run_walk = (k == 3 || (k == 0 && entries * kRunWalkMinSegment <= n_rows)) ? 1 : 0;
  }
  q.stage_bytes = stage_off;
  q.stages = (uint8_t)(opts && opts->stages ? opts->stages : 4);
  q.ncw = (uint8_t)ncw;
  if (q.stages < 1 || q.stages > 8) return set_error(CQ_ERR_INVALID_ARG, "stages must be in 1..8");
  auto& aux = P->aux;
  // ---- predicates
  // Clauses of the conjunctive form (Section 5 AND / OR / NOT): a predicate
  // with or_group 0 is a clause alone, the predicates of one nonzero group
  // share a clause.  Only a plain conjunct (a clause of one predicate, not
  // negated) restricts every passing row, so only such predicates narrow a
  // key's domain or remap its digits below.
  q.n_preds = (uint8_t)plan->n_preds;
  std::vector<int> clause_of(plan->n_preds, -1), clause_size;
  for (uint32_t i = 0; i < plan->n_preds; ++i) {
    const uint32_t g = plan->preds[i].or_group;
    if (g)
      for (uint32_t j = 0; j < i; ++j)
        if (plan->preds[j].or_group == g) {
          clause_of[i] = clause_of[j];
          break;
        }
    if (clause_of[i] < 0) {
      clause_of[i] = (int)clause_size.size();
      clause_size.push_back(0);
    }
    clause_size[clause_of[i]]++;
  }
  auto plain_conjunct = [&](uint32_t i) { return clause_size[clause_of[i]] == 1 && !plan->preds[i].negate; };
  std::vector<int> in_pred_of_col(q.n_cols, -1);
  std::vector<int> in_count(q.n_cols, 0);
  for (uint32_t i = 0; i < plan->n_preds; ++i) {
    const cq_predicate& p = plan->preds[i];
    const int ci = slot[p.col];
    const PlanCol& pc = tcols[p.col];
    const ColDesc& cd = q.cols[ci];
    PredDesc& d = q.preds[i];
    d.col = (uint8_t)ci;
    d.neg = p.negate ? 1 : 0;
    d.clause = 0;
    if (p.op < CQ_LT || p.op > CQ_IN) return set_error(CQ_ERR_INVALID_ARG, "predicate %u: bad op %d", i, p.op);
    if (is_dict(pc)) {
      const cq_column* dc = pc.src;
      const uint32_t need = p.op == CQ_IN ? 0u : (p.op == CQ_BETWEEN ? 2u : 1u);
      if (p.n_strs < need || (p.n_strs && !p.strs))
        return set_error(CQ_ERR_INVALID_ARG, "predicate %u on a dictionary column needs string literals", i);
      auto lb = [&](uint32_t k) { return dict_bound(dc, p.strs[k], lit_len(p, k), false); };
      auto ub = [&](uint32_t k) { return dict_bound(dc, p.strs[k], lit_len(p, k), true); };
      RawMap m{false, 0, 0, (i128)dc->n_entries - 1};
      switch (p.op) {
        case CQ_LT: set_range(d, 0, (i128)lb(0) - 1, m); break;
        case CQ_LE: set_range(d, 0, (i128)ub(0) - 1, m); break;
        case CQ_GT: set_range(d, ub(0), m.rmax, m); break;
        case CQ_GE: set_range(d, lb(0), m.rmax, m); break;
        case CQ_EQ: {
          const uint32_t a = lb(0), b = ub(0);
          if (a < b) set_range(d, a, a, m); else d.kind = PK_FALSE;
          break;
        }
        case CQ_NE: {
          const uint32_t a = lb(0), b = ub(0);
          if (a < b) { d.kind = PK_NE; d.lo = a; } else d.kind = PK_TRUE;
          break;
        }
        case CQ_BETWEEN: set_range(d, lb(0), (i128)ub(1) - 1, m); break;
        case CQ_IN: {
          std::vector<int64_t> codes;
          for (uint32_t k = 0; k < p.n_strs; ++k) {
            const uint32_t a = lb(k), b = ub(k);
            if (a < b) codes.push_back(a);
          }
          set_members(d, codes, aux);
          if (plain_conjunct(i)) {
            in_pred_of_col[ci] = (int)i;
            in_count[ci]++;
          }
          break;
        }
      }
      continue;
    }
    if (p.n_strs) return set_error(CQ_ERR_INVALID_ARG, "predicate %u: string literal on an integer column", i);
    const RawMap m = raw_map(pc, cd.raw_is_offset);
    switch (p.op) {
      case CQ_LT: set_range(d, LLONG_MIN, (i128)p.lo - 1, m); break;
      case CQ_LE: set_range(d, LLONG_MIN, p.lo, m); break;
      case CQ_GT: set_range(d, (i128)p.lo + 1, LLONG_MAX, m); break;
      case CQ_GE: set_range(d, p.lo, LLONG_MAX, m); break;
      case CQ_EQ: set_range(d, p.lo, p.lo, m); break;
      case CQ_BETWEEN: set_range(d, p.lo, p.hi, m); break;
      case CQ_NE: {
        const i128 r = (i128)p.lo - m.base;
        if (r < m.rmin || r > m.rmax) d.kind = PK_TRUE;
        else { d.kind = PK_NE; d.lo = (int64_t)r; }
        break;
      }
      case CQ_IN: {
        if (p.n_in && !p.in_ints) return set_error(CQ_ERR_INVALID_ARG, "predicate %u: NULL IN list", i);
        std::vector<int64_t> vals;
        for (uint32_t k = 0; k < p.n_in; ++k) {
          const i128 r = (i128)p.in_ints[k] - m.base;
          if (r >= m.rmin && r <= m.rmax) vals.push_back((int64_t)r);
        }
        set_members(d, vals, aux);
        if (plain_conjunct(i)) {
          in_pred_of_col[ci] = (int)i;
          in_count[ci]++;
        }
        break;
      }
    }
  }
  // ---- 32-bit evaluation where the column's raw values fit int32
  // a column whose raw values the kernel may read in 32 bits
  auto narrow_col = [&](const ColDesc& cd, const PlanCol& pc) {
    switch (cd.enc) {
      case ENC_PLAIN: return !cd.v64;
      case ENC_PACKED: return cd.raw_is_offset && cd.bw <= 31;
      case ENC_DICT: return cd.bw <= 31;
      case ENC_RLE: return !cd.v64;
      case ENC_INDEX: return !cd.v64 && pc.base >= INT_MIN && pc.base <= INT_MAX;
    }
    return false;
  };
  for (uint32_t i = 0; i < plan->n_preds; ++i) {
    PredDesc& d = q.preds[i];
    const ColDesc& cd = q.cols[d.col];
    const PlanCol& pc = tcols[plan->preds[i].col];
    const bool narrow = narrow_col(cd, pc);
    d.n32 = 0;
    if (!narrow) continue;
    if (d.kind == PK_RANGE) {
      const int64_t lo = std::max<int64_t>(d.lo, INT_MIN), hi = std::min<int64_t>(d.hi, INT_MAX);
      if (lo > hi) { d.kind = PK_FALSE; continue; }
      d.lo32 = (int32_t)lo;
      d.hi32 = (int32_t)hi;
      d.n32 = 1;
    } else if (d.kind == PK_NE) {
      if (d.lo < INT_MIN || d.lo > INT_MAX) { d.kind = PK_TRUE; continue; }
      d.lo32 = (int32_t)d.lo;
      d.n32 = 1;
    } else if (d.kind == PK_BITMAP && d.lo >= INT_MIN && d.hi <= INT_MAX) {
      d.lo32 = (int32_t)d.lo;
      d.hi32 = (int32_t)d.hi;
      d.n32 = 1;
    }
  }
  // a complemented constant is the other constant
  for (uint32_t i = 0; i < plan->n_preds; ++i) {
    PredDesc& d = q.preds[i];
    if (d.neg && (d.kind == PK_TRUE || d.kind == PK_FALSE)) {
      d.kind = d.kind == PK_TRUE ? PK_FALSE : PK_TRUE;
      d.neg = 0;
    }
  }
  // ---- group keys (dense mixed radix, first key most significant)
  q.n_keys = (uint8_t)plan->n_group_by;
  i128 groups = 1;
  for (uint32_t k = 0; k < plan->n_group_by; ++k) {
    const int ci = slot[plan->group_by[k]];
    const PlanCol& pc = tcols[plan->group_by[k]];
    const ColDesc& cd = q.cols[ci];
    KeyDesc& kd = q.keys[k];
    kd.col = (uint8_t)ci;
    const int ip = in_pred_of_col[ci];
    if (ip >= 0 && in_count[ci] == 1 && q.preds[ip].kind == PK_BITMAP) {
      // an IN list on the key: digits are ranks of the listed values
      const PredDesc& pd = q.preds[ip];
      kd.remap = 1;
      kd.kmin = pd.lo;
      kd.aux_off = pd.aux_off;
      kd.aux_len = pd.aux_len;
      kd.prefix_off = (uint32_t)aux.size();
      uint32_t run = 0;
      std::vector<int64_t> members;
      for (uint32_t w = 0; w < pd.aux_len; ++w) {
        aux.push_back(run);
        const uint32_t bits = aux[pd.aux_off + w];
        run += (uint32_t)__builtin_popcount(bits);
        for (int b = 0; b < 32; ++b)
          if ((bits >> b) & 1u) members.push_back(pd.lo + (int64_t)w * 32 + b);
      }
      kd.card = run;
      if (aux.size() & 1) aux.push_back(0);
      kd.list_off = (uint32_t)aux.size();
      for (int64_t v : members) {
        aux.push_back((uint32_t)(uint64_t)v);
        aux.push_back((uint32_t)((uint64_t)v >> 32));
      }
    } else {
      i128 lo, hi;
      if (is_dict(pc)) {
        lo = pc.stats.min_raw;
        hi = pc.stats.max_raw;
      } else if (cd.raw_is_offset) {
        lo = pc.stats.min_raw;
        hi = pc.stats.max_raw;
      } else {
        lo = pc.stats.min_val;
        hi = pc.stats.max_val;
      }
      // a range predicate on the key column narrows its domain
      for (uint32_t i = 0; i < plan->n_preds; ++i) {
        const PredDesc& pd = q.preds[i];
        if (pd.col != ci || !plain_conjunct(i)) continue;
        if (pd.kind == PK_RANGE) { lo = std::max(lo, (i128)pd.lo); hi = std::min(hi, (i128)pd.hi); }
        if (pd.kind == PK_BITMAP) { lo = std::max(lo, (i128)pd.lo); hi = std::min(hi, (i128)pd.hi); }
      }
      if (hi < lo) { lo = 0; hi = 0; }
      const i128 card = hi - lo + 1;
      if (card > ((i128)1 << 62))
        return set_error(CQ_ERR_UNSUPPORTED, "group-by column %u spans %.3g values; key domains are limited to 2^62",
                         plan->group_by[k], (double)card);
      kd.kmin = (int64_t)lo;
      kd.card = (uint64_t)card;
    }
    if (kd.card == 0) kd.card = 1;
    kd.n32 = (narrow_col(cd, pc) && kd.kmin >= -(1ll << 30) && kd.kmin <= (1ll << 30) && kd.card <= (1ull << 32)) ? 1 : 0;
    groups *= (i128)kd.card;
    if (groups > ((i128)1 << 62))
      return set_error(CQ_ERR_UNSUPPORTED, "the group-by key domain exceeds 2^62 groups");
  }
  uint64_t stride = 1;
  for (int k = (int)plan->n_group_by - 1; k >= 0; --k) {
    q.keys[k].stride = stride;
    stride *= q.keys[k].card;
  }
  // Key domains above 2^24 groups keep their groups in a global hash table
  // of packed 64-bit keys (a single query only; batches keep dense domains)
  q.ghash = groups > (i128)kDenseMaxGroups ? 1 : 0;
  if (q.ghash) {
    if (batch)
      return set_error(CQ_ERR_UNSUPPORTED,
                       "the group-by key domain (%.3g groups) needs the global hash table, which batched queries "
                       "do not use; run the query alone",
                       (double)groups);
    uint32_t bits = 1;
    while (bits < 63 && ((i128)1 << bits) < groups) ++bits;
    q.key_bits = (uint8_t)bits;
    // initial capacity: twice the groups that can exist (at most one per
    // row), within 2^12 .. 2^22 slots unless the options name one
    const i128 est = std::min<i128>(groups, (i128)n_rows > 0 ? (i128)n_rows : 1);
    uint32_t lg = kHashMinLog2;
    while (lg < 22 && ((i128)1 << lg) < 2 * est) ++lg;
    if (opts && opts->hash_slots_log2) lg = opts->hash_slots_log2;
    set_hash_capacity(q, lg);
  } else {
    q.key_bits = 0;
    q.n_groups = (uint64_t)groups;
  }
  // ---- evaluation order and per-run evaluation (Appendix D: predicates on
  // run-length columns are tested first, once per run value).  Row mode:
  // up to kMaxPassBitmaps RLE / index predicates get a tile pass bitmap the
  // helper warp fills from the run (listed-row) values; segment mode
  // evaluates per segment.  The descriptors are reordered in place (the keys
  // above copied what they needed): pass-bitmap predicates, other RLE /
  // index predicates, the rest.
  // A clause's predicates stay adjacent, the clause ordered by its cheapest
  // member, and its last member marked: the filter ORs a clause's members,
  // then ANDs the clause in.
  {
    q.n_pbm = 0;
    int cls[kMaxPreds];
    for (uint32_t i = 0; i < plan->n_preds; ++i) {
      PredDesc& d = q.preds[i];
      const uint8_t enc = q.cols[d.col].enc;
      const bool run_col = enc == ENC_RLE || enc == ENC_INDEX;
      d.pbm = 0xFF;
      if (run_col && !q.seg_mode && d.kind != PK_TRUE && d.kind != PK_FALSE && q.n_pbm < kMaxPassBitmaps)
        d.pbm = q.n_pbm++;
      cls[i] = d.pbm != 0xFF ? 0 : run_col ? 1 : 2;
    }
    std::vector<int> ccls(clause_size.size(), 3);
    for (uint32_t i = 0; i < plan->n_preds; ++i) ccls[clause_of[i]] = std::min(ccls[clause_of[i]], cls[i]);
    PredDesc sorted[kMaxPreds];
    uint32_t k = 0;
    for (int c = 0; c < 3; ++c)
      for (size_t cl = 0; cl < clause_size.size(); ++cl) {
        if (ccls[cl] != c) continue;
        const uint32_t first = k;
        for (int m = 0; m < 3; ++m)
          for (uint32_t i = 0; i < plan->n_preds; ++i)
            if (clause_of[i] == (int)cl && cls[i] == m) sorted[k++] = q.preds[i];
        for (uint32_t j = first; j < k; ++j)
          sorted[j].clause = k - first == 1 ? PC_ALONE : (j + 1 == k ? PC_LAST : PC_MEMBER);
      }
    for (uint32_t i = 0; i < k; ++i) q.preds[i] = sorted[i];
  }
  // ---- table shape and flush period
  q.flush_rows = 1u << 20;
  // a run walk flushes its shared table once, after all of a launch's rows
  if (q.run_walk) q.flush_rows = (uint32_t)(n_rows < kLaunchRows ? n_rows : kLaunchRows);
  // a SUM whose values are small enough for a 32-bit shared word over a
  // flush period of at least 2^18 rows shortens the period to fit it
  for (uint32_t i = 0; i < plan->n_aggs && !q.run_walk; ++i) {
    const cq_aggregate& a = plan->aggs[i];
    if ((a.op != CQ_SUM && a.op != CQ_AVG) || a.expr != CQ_EXPR_NONE) continue;
    const PlanCol& pc = tcols[a.col];
    if (pc.enc == ENC_INDEX) continue;
    const ColDesc& cd = q.cols[slot[a.col]];
    i128 lo, hi;
    if (cd.raw_is_offset) { lo = pc.stats.min_raw; hi = pc.stats.max_raw; }
    else { lo = pc.stats.min_val; hi = pc.stats.max_val; }
    const i128 bound = std::max<i128>(hi < 0 ? -hi : hi, lo < 0 ? -lo : lo) + 1;
    const i128 limit = lo >= 0 ? ((i128)1 << 32) : ((i128)1 << 31);
    uint32_t f = 1u << 20;
    while (f > (1u << 18) && bound * (i128)f >= limit) f >>= 1;
    if (bound * (i128)f < limit && f < q.flush_rows) q.flush_rows = f;
  }
  if (q.flush_rows < tile) q.flush_rows = tile;
  // ---- aggregates
  uint32_t n_all = plan->n_aggs;       // user aggregates, then hidden SUM companions of VAR / STD
  uint32_t sw = 0, sw32 = 1, gw = 1;   // 32-bit word 0 is COUNT
  q.has_index_agg = 0;
  // SUM / AVG (and the hidden SUM of a VAR / STD): accumulator layout
  auto plan_sum = [&](AggDesc& d, const PlanCol& pc, const ColDesc& cd, bool idx) {
    d.kind = idx ? AK_ISUM : AK_SUM;
    i128 bound;
    if (idx) {
      bound = (i128)pc.stats.max_abs_val + (pc.base < 0 ? -(i128)pc.base : (i128)pc.base);
      d.base = pc.base;
    } else if (cd.raw_is_offset && pc.enc == ENC_PACKED) {
      bound = (i128)std::max<int64_t>(pc.stats.max_raw, 0);
      d.base = pc.base;
    } else {
      bound = pc.stats.max_abs_val;
      d.base = 0;
    }
    d.wide = bound * (i128)q.flush_rows >= ((i128)1 << 62) ? 1 : 0;
    // raw values small enough to be summed across a warp batch in 32 bits
    i128 rlo, rhi;
    if (cd.raw_is_offset) { rlo = pc.stats.min_raw; rhi = pc.stats.max_raw; }
    else { rlo = pc.stats.min_val; rhi = pc.stats.max_val; }
    // a warp reduces up to 128 values (4 per lane) in 32 bits
    d.red32 = (!idx && !d.wide && rlo > -((i128)1 << 24) && rhi < ((i128)1 << 24)) ? 1 : 0;
    d.ubits = 0;
    if (d.red32 && rlo >= 0) {
      uint8_t b = 1;
      while (((i128)1 << b) <= rhi) ++b;
      d.ubits = b;
    }
    d.n32 = (d.red32 && narrow_col(cd, pc)) ? 1 : 0;
    {
      const i128 b = std::max<i128>(rhi < 0 ? -rhi : rhi, rlo < 0 ? -rlo : rlo) + 1;
      const i128 limit = rlo >= 0 ? ((i128)1 << 32) : ((i128)1 << 31);
      d.s32 = (!idx && b * (i128)q.flush_rows < limit) ? (rlo >= 0 ? 1 : 2) : 0;
      // else, row mode, inputs in [0, 2^24): two 32-bit limb words, the low
      // kSplitBits bits and the rest, each updated without a returned value;
      // a flush period of at most 2^20 rows keeps both below 2^32
      if (!d.s32 && !idx && !q.seg_mode && rlo >= 0 && rhi < ((i128)1 << 24) && q.flush_rows <= (1u << 20))
        d.s32 = 3;
    }
    if (d.s32) {
      d.sw32 = (uint8_t)sw32;
      sw32 += d.s32 == 3 ? 2 : 1;
    } else {
      d.sw = (uint8_t)sw;
      sw += d.wide ? 2 : 1;
    }
    d.gw = gw;
    gw += 3;
  };
  for (uint32_t i = 0; i < plan->n_aggs; ++i) {
    const cq_aggregate& a = plan->aggs[i];
    AggDesc& d = q.aggs[i];
    d.op = (uint8_t)a.op;
    d.out_kind = a.op == CQ_COUNT ? 1 : ((a.op == CQ_AVG || a.op >= CQ_VAR_POP) ? 2 : 0);
    if (a.op == CQ_COUNT) {
      d.kind = AK_COUNT;
      continue;
    }
    const int ci = slot[a.col];
    const PlanCol& pc = tcols[a.col];
    const ColDesc& cd = q.cols[ci];
    d.col = (uint8_t)ci;
    if (a.expr != CQ_EXPR_NONE) {
      // position-wise arithmetic on two columns (Section 6): the range of
      // the result by interval arithmetic on the columns' value ranges; it
      // must stay within int64, accumulated in 64-bit (or 128-bit) words
      const PlanCol& pc2 = tcols[a.col2];
      const i128 l1 = pc.stats.min_val, h1 = pc.stats.max_val, l2 = pc2.stats.min_val, h2 = pc2.stats.max_val;
      i128 lo, hi;
      if (a.expr == CQ_EXPR_ADD) {
        lo = l1 + l2;
        hi = h1 + h2;
      } else if (a.expr == CQ_EXPR_SUB) {
        lo = l1 - h2;
        hi = h1 - l2;
      } else {
        const i128 p[4] = {l1 * l2, l1 * h2, h1 * l2, h1 * h2};
        lo = std::min(std::min(p[0], p[1]), std::min(p[2], p[3]));
        hi = std::max(std::max(p[0], p[1]), std::max(p[2], p[3]));
      }
      if (lo < (i128)LLONG_MIN || hi > (i128)LLONG_MAX)
        return set_error(CQ_ERR_UNSUPPORTED, "aggregate %u: the expression's values may leave the int64 range", i);
      d.expr = (uint8_t)a.expr;
      d.col2 = (uint8_t)slot[a.col2];
      d.base = 0;
      d.red32 = d.ubits = d.n32 = d.s32 = d.w32 = 0;
      d.sw = (uint8_t)sw;
      d.gw = gw;
      if (a.op == CQ_SUM || a.op == CQ_AVG) {
        const i128 bound = std::max<i128>(hi, -lo);
        d.kind = AK_SUM;
        d.wide = bound * (i128)q.flush_rows >= ((i128)1 << 62) ? 1 : 0;
        sw += d.wide ? 2 : 1;
        gw += 3;
      } else {
        d.kind = a.op == CQ_MIN ? AK_MIN : AK_MAX;
        sw += 1;
        gw += 1;
      }
      continue;
    }
    const bool idx = pc.enc == ENC_INDEX;
    if (idx) q.has_index_agg = 1;
    if (a.op >= CQ_VAR_POP) {
      // VAR / STD (Section 7): the sum of squares of shifted values r (raw
      // offsets of a packed column, value - default of an index column), a
      // hidden SUM of the same r, and COUNT; a shift leaves a variance as is
      i128 bound;
      if (idx) bound = std::max<i128>((i128)pc.stats.max_val - pc.base, (i128)pc.base - pc.stats.min_val);
      else if (cd.raw_is_offset) bound = std::max<i128>(pc.stats.max_raw, -(i128)pc.stats.min_raw);
      else bound = std::max<i128>(pc.stats.max_val, -(i128)pc.stats.min_val);
      if (bound >= ((i128)1 << 31))
        return set_error(CQ_ERR_UNSUPPORTED, "aggregate %u: VAR/STD take values within +-2^31 of the column's base", i);
      if (n_all >= (uint32_t)kMaxAggs)
        return set_error(CQ_ERR_INVALID_ARG, "plan exceeds 16 aggregates counting those VAR/STD add");
      d.kind = idx ? AK_ISUM2 : AK_SUM2;
      d.base = idx ? pc.base : 0;
      d.wide = bound * bound * (i128)q.flush_rows >= ((i128)1 << 62) ? 1 : 0;
      d.red32 = d.ubits = d.n32 = d.s32 = d.w32 = 0;
      d.sw = (uint8_t)sw;
      sw += d.wide ? 2 : 1;
      d.gw = gw;
      gw += 3;
      d.pair = (uint8_t)n_all;
      AggDesc& c = q.aggs[n_all++];
      memset(&c, 0, sizeof(c));
      c.op = CQ_SUM;
      c.col = (uint8_t)ci;
      plan_sum(c, pc, cd, idx);
      continue;
    }
    if (a.op == CQ_SUM || a.op == CQ_AVG) {
      plan_sum(d, pc, cd, idx);
    } else {  // MIN / MAX
      i128 rlo, rhi;
      if (idx || cd.raw_is_offset) { rlo = pc.stats.min_raw; rhi = pc.stats.max_raw; }
      else { rlo = pc.stats.min_val; rhi = pc.stats.max_val; }
      d.w32 = (rlo >= (i128)INT_MIN && rhi <= (i128)INT_MAX) ? 1 : 0;
      d.n32 = (d.w32 && !idx && narrow_col(cd, pc)) ? 1 : 0;
      // value: a 32-bit word when it fits, else a 64-bit one; index
      // columns add a 32-bit listed count
      d.sw = (uint8_t)sw;
      d.sw32 = (uint8_t)sw32;
      if (d.w32) sw32 += 1; else sw += 1;
      if (idx) {
        d.kind = a.op == CQ_MIN ? AK_IMIN : AK_IMAX;
        d.base = pc.base;
        sw32 += 1;
        d.gw = gw;
        gw += 2;
      } else {
        d.kind = a.op == CQ_MIN ? AK_MIN : AK_MAX;
        d.base = (cd.raw_is_offset && pc.enc == ENC_PACKED) ? pc.base : 0;
        d.gw = gw;
        gw += 1;
      }
    }
  }
  q.n_aggs = (uint8_t)n_all;
  q.n_sw = (uint8_t)sw;
  q.n_sw32 = (uint8_t)sw32;
  q.n_gw = (uint8_t)gw;
  // ---- shared-memory group table: dense bins when the whole domain fits
  uint32_t slots = opts && opts->table_slots ? opts->table_slots : 1024;
  if (slots & (slots - 1)) return set_error(CQ_ERR_INVALID_ARG, "table_slots must be a power of two");
  const uint64_t dense_cap = 4096;
  if (q.n_groups <= dense_cap && !q.ghash) {
    q.table_dense = 1;
    q.table_slots = (uint32_t)q.n_groups;
  } else {
    q.table_dense = 0;
    q.table_slots = slots;
  }
  // ---- fit shared memory: fewer stages, then fewer slots
  q.aux_words = (uint32_t)aux.size();
  for (;;) {
    q.smem_bytes = 0;
    const size_t need = query_kernel_smem(q);
    if (need <= smem_limit) {
      q.smem_bytes = (uint32_t)need;
      break;
    }
    if (!q.seg_mode && q.stages > 2) { q.stages--; continue; }
    if (!q.table_dense && q.table_slots > 128) { q.table_slots /= 2; continue; }
    *no_fit = true;
    return set_error(CQ_ERR_UNSUPPORTED, "query does not fit in %zu bytes of shared memory (tile_rows %u)",
                     smem_limit, tile);
  }
  // grow the hash table into the shared memory left over (fewer flushes)
  if (!q.table_dense && !(opts && opts->table_slots)) {
    while (q.table_slots < 4096) {
      q.table_slots *= 2;
      if (query_kernel_smem(q) > smem_limit) {
        q.table_slots /= 2;
        break;
      }
    }
    q.smem_bytes = (uint32_t)query_kernel_smem(q);
  }
  // ncw 8 marks the two-CTA row shape; segment mode runs three (two) CTAs per
  // SM whenever its shared memory fits a third (half) of an SM
  P->ctas_per_sm = (!q.seg_mode && ncw == 8) ? 2 : 1;
  if (q.seg_mode && smem_limit <= ctx->smem_two) P->ctas_per_sm = smem_limit <= ctx->smem_three ? 3 : 2;
  P->grid_ctas = opts ? opts->grid_ctas : 0u;
  // (aggregates over expressions run the generic row kernel in row mode)
  bool has_expr = false;
  for (uint32_t i = 0; i < plan->n_aggs; ++i) has_expr = has_expr || plan->aggs[i].expr != CQ_EXPR_NONE;
  P->generic = (opts && opts->kernel == 1) || has_expr;
  P->row_fn = nullptr;
  // ---- run lines (grouping on runs, Section 7): when key 0 is an RLE column
  // whose runs are long next to the table, the specialised row kernel gives
  // every run of it a line of the shared table (slot = line * width + the
  // other keys' digits) instead of hashing the group id
  q.line_mode = 0;
  if (!batch && !q.seg_mode && !q.ghash && !q.table_dense && q.n_keys >= 1 && !P->generic && jit_enabled() &&
      q.cols[q.keys[0].col].enc == ENC_RLE) {
    const ColDesc& kc = q.cols[q.keys[0].col];
    const uint64_t inner = q.keys[0].stride;
    // (the lines' key digits live in the table's unused key words: 8 bytes a
    // line within 4 bytes a slot, so at most table_slots / 2 lines)
    uint32_t lg = 0;
    while (lg < 16 && (2ull << lg) * inner <= q.table_slots && (2ull << lg) * 2 <= q.table_slots) ++lg;
    const uint64_t lines = 1ull << lg;
    // runs a tile holds on average, plus the one it starts in
    const double per_tile = (double)tile * (double)kc.n / (double)(n_rows ? n_rows : 1) + 1.0;
    if (lines * inner <= q.table_slots && (double)lines >= 2.0 * per_tile) {
      q.line_mode = 1;
      q.line_log2 = (uint8_t)lg;
      q.line_slot = kc.bslot;
      q.line_inner = (uint32_t)inner;
      uint32_t p2 = 1;
      while (p2 < 32 && inner % (2 * p2) == 0) p2 *= 2;
      q.line_swz = p2 - 1;
    }
  }
  // ---- outputs
  q.n_out = plan->n_group_by + plan->n_aggs;
  P->out_kind.clear();
  P->out_key_col.clear();
  for (uint32_t k = 0; k < plan->n_group_by; ++k) {
    q.out_is_key[k] = 1;
    q.out_index[k] = (uint8_t)k;
    P->out_kind.push_back(0);
    P->out_key_col.push_back((int)plan->group_by[k]);
  }
  for (uint32_t i = 0; i < plan->n_aggs; ++i) {
    q.out_is_key[plan->n_group_by + i] = 0;
    q.out_index[plan->n_group_by + i] = (uint8_t)i;
    P->out_kind.push_back(q.aggs[i].out_kind);
    P->out_key_col.push_back(-1);
  }
  return CQ_OK;
}

// Plan the query, trying kernel shapes in order of preference until one fits
// in shared memory (the order is given where the shapes are listed below);
// tiles halve down to 1024 rows.  Options pin the tile size (smaller ones are
// tried when it does not fit) and / or the CTAs per SM.
static int plan_query(const std::vector<PlanCol>& tcols, uint64_t n_rows, const cq_plan* plan_in,
                      const cq_exec_options* opts, const cq_ctx* ctx, Planned* P, size_t batch_limit = 0) {
  if (!plan_in) return set_error(CQ_ERR_INVALID_ARG, "plan is NULL");
  // a filter program becomes its conjunctive form (cq_filter.cu)
  NormFilter nf;
  const int nrc = normalize_filter(plan_in, &nf);
  if (nrc != CQ_OK) return nrc;
  const cq_plan* plan = &nf.plan;
  const uint32_t want_tile = opts ? opts->tile_rows : 0;
  const uint32_t want_ctas = opts ? opts->ctas_per_sm : 0;
  if (want_tile && (want_tile < 1024 || want_tile > 8192 || (want_tile & (want_tile - 1))))
    return set_error(CQ_ERR_INVALID_ARG, "tile_rows must be 1024, 2048, 4096 or 8192");
  if (want_ctas > 3) return set_error(CQ_ERR_INVALID_ARG, "ctas_per_sm must be 0, 1, 2 or 3 (3: segment mode)");
  if (opts && opts->kernel > 3)
    return set_error(CQ_ERR_INVALID_ARG, "kernel must be 0 (default), 1 (generic row kernel), 2 (segment mode by "
                                         "tiles) or 3 (segment mode by runs)");
  if (opts && opts->hash_slots_log2 && (opts->hash_slots_log2 < kHashMinLog2 || opts->hash_slots_log2 > kHashMaxLog2))
    return set_error(CQ_ERR_INVALID_ARG, "hash_slots_log2 must be 0 or in %u..%u", kHashMinLog2, kHashMaxLog2);
  // segment mode when every referenced column is RLE or index-encoded
  bool seg = true;
  auto look = [&](uint32_t c) {
    if (c < tcols.size() && tcols[c].enc != ENC_RLE && tcols[c].enc != ENC_INDEX) seg = false;
  };
  for (uint32_t i = 0; i < plan->n_preds && plan->preds; ++i) look(plan->preds[i].col);
  for (uint32_t i = 0; i < plan->n_group_by && plan->group_by; ++i) look(plan->group_by[i]);
  for (uint32_t i = 0; i < plan->n_aggs && plan->aggs; ++i) {
    if (plan->aggs[i].op != CQ_COUNT) look(plan->aggs[i].col);
    if (plan->aggs[i].op != CQ_COUNT && plan->aggs[i].expr != CQ_EXPR_NONE) look(plan->aggs[i].col2);
  }
  struct Shape { int ncw; uint32_t tile; size_t limit; };
  std::vector<Shape> shapes;
  auto add = [&](int ncw, uint32_t first, size_t limit) {
    // a tile is 16 compute warps * 32 * GPW rows with GPW in {2, 4, 8, 16}
    // (the 24- and 28-warp shapes are listed with their own tile sizes)
    const uint32_t max_tile = 8192u;
    for (uint32_t t = want_tile ? want_tile : first; t >= 1024; t /= 2)
      if (t <= max_tile) shapes.push_back({ncw, t, limit});
  };
  if (batch_limit) {
    // a batch shares one kernel shape: 16 compute warps (+ the helper warp in
    // row mode), shared memory within the batch kernel's limit, 8192- or
    // 4096-row tiles
    if (want_tile && want_tile < 4096)
      return set_error(CQ_ERR_INVALID_ARG, "batches use 4096- or 8192-row tiles");
    if (!want_tile || want_tile == 8192) shapes.push_back({16, 8192u, batch_limit});
    shapes.push_back({16, 4096u, batch_limit});
  } else if (seg) {
    // three CTAs per SM when the tile fits a third of the shared memory, two
    // when it fits half, else one
    if (want_ctas == 0 || want_ctas == 3) add(16, 8192, ctx->smem_three);
    if (want_ctas != 1) add(16, 8192, ctx->smem_two);
    add(16, 8192, ctx->smem_optin);
  } else if (want_ctas == 2) {
    add(8, 8192, ctx->smem_two);
  } else {
    // more warps hide more latency: two CTAs of 16 compute warps per SM (ncw 8
    // marks the shape) when a full 8192-row tile fits half an SM, else one CTA
    // of 24 compute warps with 6144-row tiles, else one of 16 with tiles down
    // to 1024 rows
    if (want_ctas == 0 && want_tile == 0) {
      shapes.push_back({8, 8192u, ctx->smem_two});
      shapes.push_back({28, 7168u, ctx->smem_optin});
      shapes.push_back({24, 6144u, ctx->smem_optin});
    }
    add(16, 8192, ctx->smem_optin);
  }
  int rc = CQ_ERR_UNSUPPORTED;
  for (const Shape& sh : shapes) {
    bool no_fit = false;
    rc = plan_query_tile(tcols, n_rows, plan, opts, ctx, sh.tile, sh.ncw, sh.limit, P, &no_fit, batch_limit != 0);
    if (rc == CQ_OK || !no_fit) return rc;
  }
  return rc;
}

// Byte offsets of one query's device buffers inside one allocation.
QueryBlock query_block_layout(const Planned& P, bool with_aux) {
  const QueryDesc& q = P.q;
  const uint64_t G = q.n_groups;
  const uint64_t nb = (G + 1023) / 1024;
  auto al = [](uint64_t x) { return (x + 255) / 256 * 256; };
  QueryBlock L;
  L.gacc = 0;
  L.out = L.gacc + al(8ull * q.n_gw * G);
  // hash domains: the key table and the finalize sort's buffers
  L.hkeys = L.out + al(8ull * q.n_out * G);
  L.hsort = L.hkeys + (q.ghash ? al(8ull * G) : 0);
  L.aux = L.hsort + (q.ghash ? 2 * al(8ull * G) + 2 * al(4ull * G) + al(4ull * 256 * q.sort_blocks) : 0);
  L.err = L.aux + (with_aux ? al(4ull * (P.aux.size() + 2)) : 0);
  L.cnt = L.err + 256;
  L.blk = L.cnt + 256;
  L.total = L.blk + al(4ull * (nb + 1));
  return L;
}

// Point the descriptor at the buffers of a block laid out by
// query_block_layout (aux tables at `aux_dev`).
void bind_query_block(Planned& P, uint8_t* b, const QueryBlock& L, const uint32_t* aux_dev) {
  QueryDesc& q = P.q;
  const uint64_t G = q.n_groups;
  q.gacc = reinterpret_cast<unsigned long long*>(b + L.gacc);
  for (uint32_t i = 0; i < q.n_out; ++i) q.out[i] = b + L.out + (uint64_t)i * 8 * G;
  if (q.ghash) {
    auto al = [](uint64_t x) { return (x + 255) / 256 * 256; };
    uint8_t* h = b + L.hsort;
    q.gkeys = reinterpret_cast<unsigned long long*>(b + L.hkeys);
    q.skeys[0] = reinterpret_cast<unsigned long long*>(h);
    q.skeys[1] = reinterpret_cast<unsigned long long*>(h + al(8ull * G));
    q.svals[0] = reinterpret_cast<uint32_t*>(h + 2 * al(8ull * G));
    q.svals[1] = reinterpret_cast<uint32_t*>(h + 2 * al(8ull * G) + al(4ull * G));
    q.shist = reinterpret_cast<uint32_t*>(h + 2 * al(8ull * G) + 2 * al(4ull * G));
  } else {
    q.gkeys = nullptr;
    q.skeys[0] = q.skeys[1] = nullptr;
    q.svals[0] = q.svals[1] = nullptr;
    q.shist = nullptr;
  }
  q.aux = aux_dev;
  q.aux_words = (uint32_t)P.aux.size();
  q.err = reinterpret_cast<int*>(b + L.err);
  q.err_info = reinterpret_cast<unsigned long long*>(b + L.err + 8);
  q.out_count = reinterpret_cast<unsigned long long*>(b + L.cnt);
  q.block_counts = reinterpret_cast<unsigned int*>(b + L.blk);
}

// Record in the result where its status, count and output columns live.
void attach_outputs(cq_result* r, const Planned& P) {
  r->desc = P.q;
  r->err_dev = P.q.err;
  r->count_dev = P.q.out_count;
  r->n_out = P.q.n_out;
  r->out_kind = P.out_kind;
  r->out_key_col = P.out_key_col;
  r->out_dev.assign(P.q.out, P.q.out + P.q.n_out);
}

// Carve one pool allocation into the query's device buffers and enqueue
// init -> fused kernel -> finalize on `s`.
// Row mode: resolve the kernel specialised to the query's shape (compiled on
// first use of the shape in this process).
int prepare_row_kernel(cq_ctx* ctx, Planned& P) {
  QueryDesc& q = P.q;
  if (q.seg_mode || P.generic || P.row_fn || !jit_enabled()) return CQ_OK;
  int ncw, gpw, minb;
  row_shape(q, &ncw, &gpw, &minb);
  return jit_row_kernel(q, ncw, gpw, minb, ctx->device, ctx->smem_optin, &P.row_fn);
}

static int launch_planned(cq_ctx* ctx, Planned& P, cudaStream_t s, cq_result* r) {
  QueryDesc& q = P.q;
  const int prc = prepare_row_kernel(ctx, P);
  if (prc != CQ_OK) return prc;
  clear_stale_error("a query launch");
  const QueryBlock L = query_block_layout(P, true);
  void* base = nullptr;
  cudaError_t e = pool_alloc((void**)&base, L.total, ctx->pool, s);
  if (e != cudaSuccess) return set_error(CQ_ERR_OOM, "device pool allocation of %llu bytes failed: %s", (unsigned long long)L.total, cudaGetErrorString(e));
  r->dev_block = base;
  r->dev_bytes = L.total;
  uint8_t* b = reinterpret_cast<uint8_t*>(base);
  bind_query_block(P, b, L, reinterpret_cast<const uint32_t*>(b + L.aux));
  if (!P.aux.empty()) {
    // the descriptor's aux words travel through the stream like the launch itself
    e = cudaMemcpyAsync(b + L.aux, P.aux.data(), 4 * P.aux.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "aux upload failed: %s", cudaGetErrorString(e));
  }
  const char* step = "init";
  e = launch_init_global(q, s);
  if (e == cudaSuccess && (step = "event", true)) e = cudaEventRecord(r->ev_k0, s);
  if (e == cudaSuccess && (step = "fused kernel", true)) {
    // launches of at most kLaunchRows rows, the SUM limbs folded in between
    // (CQ_LAUNCH_ROWS in the environment lowers the split, for tests)
    uint64_t rows = kLaunchRows;
    if (const char* env = getenv("CQ_LAUNCH_ROWS")) {
      const unsigned long long v = strtoull(env, nullptr, 10);
      if (v >= q.tile_rows && v < rows) rows = v;
    }
    const uint64_t chunk = rows / q.tile_rows;
    for (uint64_t t0 = 0; t0 < q.n_tiles && e == cudaSuccess; t0 += chunk) {
      QueryDesc qc = q;
      qc.tile0 = t0;
      qc.n_tiles = q.n_tiles - t0 < chunk ? q.n_tiles - t0 : chunk;
      e = launch_query(qc, s, ctx->num_sms, P.ctas_per_sm, P.grid_ctas, P.row_fn);
      if (e == cudaSuccess && t0 + chunk < q.n_tiles && (step = "fold", true)) e = launch_fold_sums(q, s);
    }
  }
  if (e == cudaSuccess && (step = "event", true)) e = cudaEventRecord(r->ev_k1, s);
  if (e == cudaSuccess && (step = "finalize", true)) e = launch_finalize(q, s);
  if (e != cudaSuccess)
    return set_error(CQ_ERR_CUDA, "%s launch failed: %s (tile %u, %llu tiles, %llu groups, %u B shared)", step,
                     cudaGetErrorString(e), q.tile_rows, (unsigned long long)q.n_tiles,
                     (unsigned long long)q.n_groups, q.smem_bytes);
  attach_outputs(r, P);
  return CQ_OK;
}

cq_result* new_result(cq_ctx* ctx, cudaStream_t s, bool own_events) {
  cq_result* r = new cq_result;
  r->ctx = ctx;
  r->stream = s;
  r->own_events = own_events;
  if (own_events) {
    cudaEventCreate(&r->ev_start);
    cudaEventCreate(&r->ev_done);
    cudaEventCreate(&r->ev_k0);
    cudaEventCreate(&r->ev_k1);
  }
  return r;
}

void free_result(cq_result* r) {
  if (!r) return;
  if (r->dev_block) cudaFreeAsync(r->dev_block, r->stream);
  for (void* p : r->extra_dev) cudaFreeAsync(p, r->stream);
  if (r->own_events) {
    if (r->ev_start) cudaEventDestroy(r->ev_start);
    if (r->ev_done) cudaEventDestroy(r->ev_done);
    if (r->ev_k0) cudaEventDestroy(r->ev_k0);
    if (r->ev_k1) cudaEventDestroy(r->ev_k1);
  }
  delete r;
}

// Launch one planned query with the one-query kernels (the serving loop's
// path for a batch of one); the result holds the table's columns.
int launch_solo(cq_table* table, Planned& P, cudaStream_t s, cq_result** out) {
  cq_ctx* ctx = table->ctx;
  cq_result* r = new_result(ctx, s, true);
  cudaEventRecord(r->ev_start, s);
  const int rc = launch_planned(ctx, P, s, r);
  if (rc != CQ_OK) {
    free_result(r);
    return rc;
  }
  if (P.q.ghash) r->retry.reset(new Planned(P));   // cq_result_wait may relaunch it larger
  for (int kc : P.out_key_col) r->key_cols.push_back(kc >= 0 ? table->cols[kc] : nullptr);
  for (cq_column* c : table->cols) c->refs++;
  r->held_cols = table->cols;
  cudaEventRecord(r->ev_done, s);
  *out = r;
  return CQ_OK;
}

// Plan one query for a launch of its own (cq_query_run's planner).
int plan_solo_query(cq_table* table, const cq_plan* plan, Planned* P) {
  if (!table) return set_error(CQ_ERR_INVALID_ARG, "NULL table");
  std::vector<PlanCol> cols;
  cols.reserve(table->cols.size());
  for (cq_column* c : table->cols) cols.push_back(view_of(c));
  return plan_query(cols, table->n_rows, plan, nullptr, table->ctx, P);
}

// Plan one query of a batch (see plan_query): the shared kernel shape, tiles
// of `tile_rows` rows (0 = the mode's default), shared memory within
// `smem_limit` bytes.
int plan_batch_query(cq_table* table, const cq_plan* plan, uint32_t tile_rows, size_t smem_limit, Planned* P) {
  if (!table) return set_error(CQ_ERR_INVALID_ARG, "NULL table");
  if (table->n_rows > kLaunchRows)
    return set_error(CQ_ERR_UNSUPPORTED, "batched queries take tables of at most 2^31 rows (%llu given); run it alone",
                     (unsigned long long)table->n_rows);
  std::vector<PlanCol> cols;
  cols.reserve(table->cols.size());
  for (cq_column* c : table->cols) cols.push_back(view_of(c));
  cq_exec_options o;
  memset(&o, 0, sizeof(o));
  o.tile_rows = tile_rows;
  return plan_query(cols, table->n_rows, plan, &o, table->ctx, P, smem_limit);
}

}  // namespace cq

// ====================================================================== queries
extern "C" int cq_query_run_ex(cq_table* table, const cq_plan* plan, const cq_exec_options* opts, void* cuda_stream,
                               cq_result** out) {
  clear_error();
  if (!table || !out) return set_error(CQ_ERR_INVALID_ARG, "NULL table or out");
  *out = nullptr;
  cq_ctx* ctx = table->ctx;
  CQ_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = cuda_stream ? reinterpret_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  const int mode = opts ? opts->mode : CQ_EXEC_FUSED;
  if (mode != CQ_EXEC_FUSED && mode != CQ_EXEC_DECOMPRESS_THEN_SCAN)
    return set_error(CQ_ERR_INVALID_ARG, "unknown execution mode %d", mode);
  std::vector<PlanCol> cols;
  for (cq_column* c : table->cols) cols.push_back(view_of(c));
  cq_result* r = new_result(ctx, s, true);
  cudaEventRecord(r->ev_start, s);
  if (mode == CQ_EXEC_DECOMPRESS_THEN_SCAN) {
    // expand every referenced column to a flat int64 array first
    std::vector<bool> used(cols.size(), false);
    if (plan) {
      for (uint32_t i = 0; i < plan->n_preds && plan->preds; ++i) if (plan->preds[i].col < cols.size()) used[plan->preds[i].col] = true;
      for (uint32_t i = 0; i < plan->n_group_by && plan->group_by; ++i) if (plan->group_by[i] < cols.size()) used[plan->group_by[i]] = true;
      for (uint32_t i = 0; i < plan->n_aggs && plan->aggs; ++i) {
        const cq_aggregate& a = plan->aggs[i];
        if (a.op != CQ_COUNT && a.col < cols.size()) used[a.col] = true;
        if (a.op != CQ_COUNT && a.expr != CQ_EXPR_NONE && a.col2 < cols.size()) used[a.col2] = true;
      }
    }
    for (size_t i = 0; i < cols.size(); ++i) {
      if (!used[i]) continue;
      void* flat = nullptr;
      cudaError_t e = pool_alloc((void**)&flat, pad16(table->n_rows * 8) + 16, ctx->pool, s);
      if (e != cudaSuccess) {
        free_result(r);
        return set_error(CQ_ERR_OOM, "flat column allocation failed: %s", cudaGetErrorString(e));
      }
      r->extra_dev.push_back(flat);
      e = expand_column(table->cols[i], reinterpret_cast<long long*>(flat), s, ctx->num_sms);
      if (e != cudaSuccess) {
        free_result(r);
        return set_error(CQ_ERR_CUDA, "expansion failed: %s", cudaGetErrorString(e));
      }
      PlanCol& pc = cols[i];
      pc.enc = ENC_PLAIN;
      pc.v64 = true;
      pc.vals = flat;
      pc.n = table->n_rows;
      pc.bw = 0;
      // flat values are logical values (dictionary: codes)
      if (table->cols[i]->enc == ENC_DICT) {
        pc.stats.min_val = pc.stats.min_raw;
        pc.stats.max_val = pc.stats.max_raw;
      }
    }
  }
  Planned P;
  int rc = plan_query(cols, table->n_rows, plan, opts, ctx, &P);
  if (rc == CQ_OK) rc = launch_planned(ctx, P, s, r);
  if (rc != CQ_OK) {
    free_result(r);
    return rc;
  }
  if (P.q.ghash) r->retry.reset(new Planned(P));   // cq_result_wait may relaunch it larger
  for (int kc : P.out_key_col) r->key_cols.push_back(kc >= 0 ? table->cols[kc] : nullptr);
  for (cq_column* c : table->cols) c->refs++;   // results keep their columns' dictionaries alive
  r->held_cols = table->cols;
  cudaEventRecord(r->ev_done, s);
  *out = r;
  return CQ_OK;
}

extern "C" int cq_query_run(cq_table* table, const cq_plan* plan, void* cuda_stream, cq_result** out) {
  return cq_query_run_ex(table, plan, nullptr, cuda_stream, out);
}

// Message for a device-side status, with the detail the kernel recorded.
static int report_status(cq_result* r) {
  const int err = r->status;
  if (!err) return CQ_OK;
  unsigned long long st[4] = {0, 0, 0, 0};
  cudaMemcpy(st, r->err_dev, sizeof(st), cudaMemcpyDeviceToHost);
  const unsigned long long what = st[1] & 0xFF, idx = st[1] >> 8;
  if (err == CQ_ERR_OVERFLOW)
    return set_error(err, "SUM of aggregate %llu does not fit int64 (dense group %llu)", idx, st[2]);
  if (err == CQ_ERR_TIMEOUT) return set_error(err, "a bounded device wait gave up");
  if (err == CQ_ERR_TABLE_FULL)
    return set_error(err, "the global group hash table (%llu slots) is full at key %llu", st[2], st[3]);
  if (err == CQ_ERR_INVALID_ARG && what == 1)
    return set_error(err, "group-by key %llu at row %llu has value %lld outside its recorded domain", idx, st[2],
                     (long long)st[3]);
  if (err == CQ_ERR_INVALID_ARG && what == 2)
    return set_error(err, "bitmap column %llu: boundary %llu lies before tile row %llu (corrupt cursor)", idx,
                     st[3], st[2]);
  if (err == CQ_ERR_INVALID_ARG && what == 4)
    return set_error(err, "shared group-table slot %llu was counted without a valid key (%llu); its updates were "
                     "dropped", st[2], st[3]);
  return set_error(err, "device status %d", err);
}

extern "C" int cq_result_wait(cq_result* r, uint64_t timeout_us) {
  clear_error();
  if (!r) return set_error(CQ_ERR_INVALID_ARG, "NULL result");
  if (r->waited) return report_status(r);
  cudaSetDevice(r->ctx->device);
  if (timeout_us != UINT64_MAX) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t q = cudaEventQuery(r->ev_done);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return set_error(CQ_ERR_CUDA, "query failed: %s", cudaGetErrorString(q));
      const auto us = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
      if ((uint64_t)us >= timeout_us) return set_error(CQ_ERR_NOT_READY, "query still running");
      std::this_thread::yield();
    }
  }
  cudaError_t e = cudaEventSynchronize(r->ev_done);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "query failed: %s", cudaGetErrorString(e));
  unsigned long long st[4] = {0, 0, 0, 0};   // status word, then what / where / value
  unsigned long long cnt = 0;
  e = cudaMemcpy(st, r->err_dev, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&cnt, r->count_dev, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "status read-back failed: %s", cudaGetErrorString(e));
  int err = (int)(uint32_t)st[0];
  // a full global hash table: launch again with four times the slots
  while (err == CQ_ERR_TABLE_FULL && r->retry) {
    Planned& P = *r->retry;
    uint32_t lg = 0;
    while ((1ull << lg) < P.q.n_groups) ++lg;
    if (lg + 2 > kHashMaxLog2) break;
    cudaFreeAsync(r->dev_block, r->stream);
    r->dev_block = nullptr;
    set_hash_capacity(P.q, lg + 2);
    int rc = launch_planned(r->ctx, P, r->stream, r);
    if (rc != CQ_OK) return rc;
    e = cudaEventRecord(r->ev_done, r->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(r->ev_done);
    if (e == cudaSuccess) e = cudaMemcpy(st, r->err_dev, sizeof(st), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&cnt, r->count_dev, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "query failed: %s", cudaGetErrorString(e));
    err = (int)(uint32_t)st[0];
    r->retries++;
  }
  r->waited = true;
  r->n_groups = cnt;
  r->status = err;
  return report_status(r);
}

extern "C" int cq_result_num_groups(cq_result* r, uint64_t* n) {
  if (!r || !n) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  int rc = cq_result_wait(r, UINT64_MAX);
  if (rc != CQ_OK && rc != CQ_ERR_OVERFLOW) return rc;
  *n = r->n_groups;
  return rc;
}

extern "C" int cq_result_num_columns(cq_result* r, uint32_t* n) {
  if (!r || !n) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  *n = r->n_out;
  return CQ_OK;
}

extern "C" int cq_result_column_kind(cq_result* r, uint32_t out_col, uint32_t* kind) {
  if (!r || !kind || out_col >= r->n_out) return set_error(CQ_ERR_INVALID_ARG, "bad output column");
  *kind = r->out_kind[out_col];
  return CQ_OK;
}

extern "C" int cq_result_fetch(cq_result* r, uint32_t out_col, void* host_dst, uint64_t dst_bytes) {
  clear_error();
  if (!r || out_col >= r->n_out) return set_error(CQ_ERR_INVALID_ARG, "bad output column");
  int rc = cq_result_wait(r, UINT64_MAX);
  if (rc != CQ_OK) return rc;
  const uint64_t bytes = r->n_groups * 8;
  if (dst_bytes < bytes) return set_error(CQ_ERR_SIZE_MISMATCH, "destination holds %llu bytes, %llu needed", (unsigned long long)dst_bytes, (unsigned long long)bytes);
  if (bytes) CQ_CUDA(cudaMemcpy(host_dst, r->out_dev[out_col], bytes, cudaMemcpyDeviceToHost));
  return CQ_OK;
}

extern "C" int cq_result_device_column(cq_result* r, uint32_t out_col, const void** dptr) {
  if (!r || !dptr || out_col >= r->n_out) return set_error(CQ_ERR_INVALID_ARG, "bad output column");
  *dptr = r->out_dev[out_col];
  return CQ_OK;
}

extern "C" int cq_result_key_string(cq_result* r, uint32_t key_col, uint64_t row, const char** s, uint32_t* len) {
  clear_error();
  if (!r || !s || !len || key_col >= r->n_out || r->out_key_col[key_col] < 0)
    return set_error(CQ_ERR_INVALID_ARG, "output column %u is not a group key", key_col);
  const cq_column* c = r->key_cols[key_col];
  if (!c || c->enc != ENC_DICT) return set_error(CQ_ERR_INVALID_ARG, "key column is not a dictionary column");
  int rc = cq_result_wait(r, UINT64_MAX);
  if (rc != CQ_OK) return rc;
  if (row >= r->n_groups) return set_error(CQ_ERR_INVALID_ARG, "row out of range");
  long long code = 0;
  CQ_CUDA(cudaMemcpy(&code, reinterpret_cast<const long long*>(r->out_dev[key_col]) + row, 8, cudaMemcpyDeviceToHost));
  if (code < 0 || (uint64_t)code >= c->n_entries) return set_error(CQ_ERR_INVALID_ARG, "code out of range");
  *s = c->dict_bytes.data() + c->dict_offsets[code];
  *len = (uint32_t)(c->dict_offsets[code + 1] - c->dict_offsets[code]);
  return CQ_OK;
}

extern "C" int cq_result_device_time_us(cq_result* r, double* us) {
  if (!r || !us) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaEventSynchronize(r->ev_done);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "%s", cudaGetErrorString(e));
  float ms = 0.f;
  e = cudaEventElapsedTime(&ms, r->ev_start, r->ev_done);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "%s", cudaGetErrorString(e));
  *us = ms * 1000.0;
  return CQ_OK;
}

extern "C" int cq_result_kernel_time_us(cq_result* r, double* us) {
  if (!r || !us) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaEventSynchronize(r->ev_done);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "%s", cudaGetErrorString(e));
  float ms = 0.f;
  e = cudaEventElapsedTime(&ms, r->ev_k0, r->ev_k1);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "%s", cudaGetErrorString(e));
  *us = ms * 1000.0;
  return CQ_OK;
}

extern "C" int cq_result_destroy(cq_result* r) {
  clear_error();
  if (!r) return CQ_OK;
  cudaSetDevice(r->ctx->device);
  cudaStreamSynchronize(r->stream);
  std::vector<cq_column*> held = r->held_cols;
  free_result(r);
  for (cq_column* c : held) cq_column_destroy(c);
  return CQ_OK;
}

// ====================================================================== alignment
extern "C" int cq_align_segments(cq_ctx* ctx, cq_column* const* cols, uint32_t k, void* cuda_stream,
                                 int64_t* seg_ends, int64_t* ridx, uint64_t capacity, uint64_t* n_segments) {
  clear_error();
  if (!ctx || !cols || !n_segments) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  if (k == 0 || k > (uint32_t)kMaxBitmapCols) return set_error(CQ_ERR_INVALID_ARG, "k must be in 1..%d", kMaxBitmapCols);
  for (uint32_t j = 0; j < k; ++j) {
    if (!cols[j] || cols[j]->enc != ENC_RLE) return set_error(CQ_ERR_INVALID_ARG, "column %u is not RLE", j);
    if (cols[j]->n_rows != cols[0]->n_rows) return set_error(CQ_ERR_SIZE_MISMATCH, "row counts differ");
  }
  if (capacity && (!seg_ends || !ridx)) return set_error(CQ_ERR_INVALID_ARG, "NULL output buffer");
  CQ_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = cuda_stream ? reinterpret_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  const unsigned long long n_rows = cols[0]->n_rows;
  const unsigned long long n_tiles = (n_rows + 4095) / 4096;
  *n_segments = 0;
  if (n_tiles == 0) return CQ_OK;
  void* scratch = nullptr;
  CQ_CUDA(pool_alloc((void**)&scratch, 8 * n_tiles, ctx->pool, s));
  std::vector<unsigned long long> host(n_tiles);
  unsigned long long ns = 0;
  cudaError_t e = align_segments(cols, k, s, scratch, n_tiles, n_rows, reinterpret_cast<long long*>(seg_ends),
                                 reinterpret_cast<long long*>(ridx), capacity, host.data(), &ns);
  cudaFreeAsync(scratch, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "alignment failed: %s", cudaGetErrorString(e));
  *n_segments = ns;
  if (ns > capacity) return set_error(CQ_ERR_SIZE_MISMATCH, "%llu segments, capacity %llu", ns, (unsigned long long)capacity);
  return CQ_OK;
}

// ====================================================================== self-test
namespace cq {
cudaError_t launch_bounded_wait_selftest(uint64_t limit_ns, int* status, cudaStream_t s);   // cq_columns.cu
}

extern "C" int cq_selftest_bounded_wait(cq_ctx* ctx, uint32_t limit_us, int32_t* device_status) {
  clear_error();
  if (!ctx || !device_status) return set_error(CQ_ERR_INVALID_ARG, "NULL argument");
  if (limit_us == 0 || limit_us > 5000000u) return set_error(CQ_ERR_INVALID_ARG, "limit must be 1 us .. 5 s");
  CQ_CUDA(cudaSetDevice(ctx->device));
  void* d = nullptr;
  CQ_CUDA(pool_alloc((void**)&d, 16, ctx->pool, ctx->stream));
  cudaError_t e = launch_bounded_wait_selftest(1000ull * limit_us, reinterpret_cast<int*>(d), ctx->stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(d, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "self-test failed: %s", cudaGetErrorString(e));
  *device_status = h;
  return CQ_OK;
}
